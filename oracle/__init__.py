"""FP64 CPU oracle for the reduced-space Gauss-Newton-Krylov registration method
of Mang & Biros, "Constrained H1-regularization schemes for diffeomorphic image
registration" (arXiv 1503.00757).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (no kernels, headers, tables or helpers); the two
meet only in the seeded input generator ``paper_1503_00757_gb300.synth``, which
holds none of the method's arithmetic.

Everything here is plain, slow and written to be checked against the paper by
eye: FP64 numpy arrays, an own radix-2 FFT (``oracle.fft``), the spectral
operators of Sec. 3.3 / Eq. (e:project-body-force) (``oracle.spectral``), the
RK2 transport solves of Eqs. (e:state-eq-elim)-(e:inc-adj-eq-elim)
(``oracle.transport``), the reduced gradient, Gauss-Newton Hessian matvec,
PCG (Algorithm 2), Armijo line search and Newton outer loop (Algorithm 1)
(``oracle.registration``), the deformation gradient of Eq. (e:def-grad)
(``oracle.transport.defgrad``) and the nonlinear Stokes (shear control)
operators of Eqs. (e:shear-control-reg-v), (e:1st-var-reg-v-nls) and
(e:2nd-var-reg-v-nls) (``oracle.shear``).

Pins (see ``tests/test_oracle_*.py``): O(n^2) DFT sums, closed-form Fourier
symbols on single modes, projector identities, the closed-form Heun
amplification for constant velocity, exact transposition of forward and
adjoint transport, second-order convergence to an exact shift and to an exact
shear-flow solution, finite-difference checks of the gradient and the
Gauss-Newton Hessian, dense-Hessian brute force on tiny grids, and the exact
deformation gradient of a shear flow.
"""
