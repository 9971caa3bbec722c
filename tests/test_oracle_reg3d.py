"""Pins for the three-dimensional oracle (oracle/reg3d.py), CPU only.

* Spectral operators on single Fourier modes (closed forms), the projection K (div K b = 0,
  gradients removed; with a mass source the eigenvalue bv / (bw (1 + |k|^2) + bv) along k).
* Heun transport with a constant velocity on one mode: every step multiplies the mode by
  1 + z + z^2 / 2, z = -i h k~ . v (closed form).
* Reduction to two dimensions: fields constant along x3 with v3 = 0 reproduce the
  independently written 2-D oracle (oracle/registration.py): J times the x3 period 2 pi, the
  gradient and the Gauss-Newton matvec in components 1, 2, and zero in component 3.
* A genuinely 3-D problem (x3 dependence, v3 != 0): the gradient against central differences
  of J, and at a zero-residual point the Gauss-Newton matvec against central differences of
  the gradient, both converging at second order in the time step (optimize-then-discretize).
* Algorithm 1: reduction to the 2-D oracle's solve and convergence on a 3-D problem."""
import math

import numpy as np
import pytest

from oracle import reg3d as R
from oracle.registration import Registration
from oracle import spectral as S2


def _mode(shape, k, phase=0.4):
    X = R.grid_coords(shape)
    arg = sum(kc * Xc for kc, Xc in zip(k, X)) + phase
    return np.cos(arg), np.sin(arg)


@pytest.mark.parametrize("k", [(1, 0, 0), (2, -3, 1), (0, 1, 5)])
def test_grad_div_A_on_single_modes(k):
    shape = (16, 8, 16)
    c, s = _mode(shape, k)
    g = R.grad(c)
    for d in range(3):
        assert np.abs(g[d] + k[d] * s).max() < 1e-12
    v = np.stack([c, 2.0 * c, -c])
    assert np.abs(R.div(v) + (k[0] + 2 * k[1] - k[2]) * s).max() < 1e-12
    assert np.abs(R.apply_A(v) - sum(kc * kc for kc in k) * v).max() < 1e-11


def test_projection_incompressible_and_mass_source():
    rng = np.random.default_rng(0)
    shape = (8, 16, 8)
    b = rng.standard_normal((3,) + shape)
    Kb = R.apply_K(b, 1e-2, math.inf)
    assert np.abs(R.div(Kb)).max() < 1e-11 * np.abs(b).max()
    phi = rng.standard_normal(shape)
    assert np.abs(R.apply_K(R.grad(phi), 1e-2, math.inf)).max() < 1e-11 * np.abs(R.grad(phi)).max()
    assert np.array_equal(R.apply_K(b, 1e-2, 0.0), b)
    # mass source: a gradient mode along k is scaled by bv / (bw (1 + |k|^2) + bv), the
    # eigenvalue 1 - |k|^2 / (|k|^2 + bv |k|^2 / (bw (1 + |k|^2))); orthogonal modes are kept
    bv, bw, k = 1e-2, 1e-3, (1, 2, -2)
    c, s = _mode(shape, k)
    gmode = np.stack([kc * s for kc in k])
    perp = np.stack([2.0 * s, -s, 0.0 * s])  # k . (2, -1, 0) = 0
    kk = sum(kc * kc for kc in k)
    lam = bv / (bw * (1.0 + kk) + bv)
    assert np.abs(R.apply_K(gmode, bv, bw) - lam * gmode).max() < 1e-12
    assert np.abs(R.apply_K(perp, bv, bw) - perp).max() < 1e-12


def test_heun_transport_of_one_mode_closed_form():
    shape, nt, k = (8, 8, 16), 6, (1, -2, 3)
    v = np.stack([np.full(shape, 0.3), np.full(shape, -0.2), np.full(shape, 0.15)])
    c, s = _mode(shape, k, phase=0.0)
    m, gm = R.state_solve(c, v, nt)
    z = -1j * (1.0 / nt) * sum(kc * vc for kc, vc in zip(k, (0.3, -0.2, 0.15)))
    amp = (1 + z + 0.5 * z * z) ** nt
    X = R.grid_coords(shape)
    arg = sum(kc * Xc for kc, Xc in zip(k, X))
    exact = np.real(amp * np.exp(1j * arg))
    assert np.abs(m[-1] - exact).max() < 1e-12
    assert np.abs(gm[-1][0] - np.real(1j * k[0] * amp * np.exp(1j * arg))).max() < 1e-11


@pytest.mark.parametrize("beta_w", [math.inf, 0.0, 1e-3])
def test_constant_along_x3_reduces_to_the_2d_oracle(beta_w):
    n, n3, nt, bv = 16, 4, 4, 1e-2
    rng = np.random.default_rng(1)
    X1, X2 = S2.grid_coords(n, n)
    mT2 = np.exp(-((X1 - 3.0) ** 2 + (X2 - 3.2) ** 2)) + 0.5 * np.exp(-((X1 - 2.0) ** 2 + (X2 - 4.0) ** 2) / 0.5)
    mR2 = np.exp(-((X1 - 3.3) ** 2 + (X2 - 2.9) ** 2)) + 0.5 * np.exp(-((X1 - 2.2) ** 2 + (X2 - 3.7) ** 2) / 0.5)
    v2 = 0.3 * np.stack([np.sin(X2) * np.cos(X1), np.sin(X1 + 0.5) * np.cos(2 * X2)])
    vt2 = 0.2 * rng.standard_normal((2, n, n))
    lift = lambda f: np.repeat(f[..., None], n3, axis=-1)
    mT3, mR3 = lift(mT2), lift(mR2)
    v3 = np.concatenate([lift(v2), np.zeros((1, n, n, n3))])
    vt3 = np.concatenate([lift(vt2), np.zeros((1, n, n, n3))])
    P2 = Registration(mT2, mR2, nt, regnorm=S2.H1, beta_v=bv, beta_w=beta_w)
    P3 = R.Registration3D(mT3, mR3, nt, bv, beta_w)
    g2, J2 = P2.gradient(v2)
    g3, J3 = P3.gradient(v3)
    assert abs(J3 - 2 * np.pi * J2) < 1e-11 * abs(J3)
    scale = np.abs(g2).max()
    assert np.abs(g3[:2] - np.stack([lift(g2[0]), lift(g2[1])])).max() < 1e-10 * scale
    assert np.abs(g3[2]).max() < 1e-12 * scale
    H2 = P2.matvec(vt2)
    H3 = P3.matvec(vt3)
    sH = np.abs(H2).max()
    assert np.abs(H3[:2] - np.stack([lift(H2[0]), lift(H2[1])])).max() < 1e-10 * sH
    assert np.abs(H3[2]).max() < 1e-12 * sH


def _problem3d(nt, beta_w=math.inf):
    shape = (16, 8, 8)
    X1, X2, X3 = R.grid_coords(shape)
    bump = lambda a, b, c: np.exp(-((np.sin((X1 - a) / 2)) ** 2 + np.sin((X2 - b) / 2) ** 2 + np.sin((X3 - c) / 2) ** 2) * 4)
    mT = bump(3.0, 3.1, 2.9)
    mR = bump(3.2, 2.9, 3.3)
    v = 0.2 * np.stack([np.sin(X2 + X3), np.cos(X1) * np.sin(X3), np.sin(X1 - X2)])
    d = 0.1 * np.stack([np.cos(X3), np.sin(X1 + X3), np.cos(X2)])
    # the incompressible gradient is the derivative of J along divergence-free directions
    d = R.apply_K(d, 1e-2, beta_w) if np.isinf(beta_w) else d
    return R.Registration3D(mT, mR, nt, 1e-2, beta_w), v, d


@pytest.mark.parametrize("beta_w", [math.inf, 0.0])
def test_gradient_matches_finite_differences_second_order(beta_w):
    errs = []
    for nt in (2, 4, 8):
        P, v, d = _problem3d(nt, beta_w)
        g, _ = P.gradient(v)
        eps = 1e-5
        fd = (P.objective(v + eps * d)[0] - P.objective(v - eps * d)[0]) / (2 * eps)
        errs.append(abs(R.inner(g, d) - fd) / abs(fd))
    assert errs[-1] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_precond_inverts_beta_A_off_the_zero_mode():
    rng = np.random.default_rng(5)
    r = rng.standard_normal((3, 8, 16, 8))
    r -= r.mean(axis=(1, 2, 3), keepdims=True)
    assert np.abs(1e-2 * R.apply_A(R.apply_precond(r, 1e-2)) - r).max() < 1e-10 * np.abs(r).max()
    c = np.ones((3, 8, 16, 8))
    assert np.abs(R.apply_precond(c, 1e-2) - 100.0 * c).max() < 1e-9


def test_solve_reduces_to_the_2d_solve():
    """Fields constant along x3: the 3-D Algorithm 1 takes the 2-D oracle's Newton and PCG
    steps (same counts) and returns its velocity in components 1, 2 (zero in component 3)."""
    n, n3, nt = 16, 4, 4
    X1, X2 = S2.grid_coords(n, n)
    mT2 = np.exp(-((X1 - 3.0) ** 2 + (X2 - 3.2) ** 2))
    mR2 = np.exp(-((X1 - 3.4) ** 2 + (X2 - 2.9) ** 2) / 1.2)
    lift = lambda f: np.repeat(f[..., None], n3, axis=-1)
    P2 = Registration(mT2, mR2, nt, regnorm=S2.H1, beta_v=1e-2, beta_w=math.inf)
    v2, st2 = P2.solve(tol=1e-3)
    P3 = R.Registration3D(lift(mT2), lift(mR2), nt, 1e-2, math.inf)
    v3, st3 = R.solve(P3, tol=1e-3)
    assert st3["status"] == 0 and st2["status"] == 0
    assert (st3["n_newton"], st3["n_mv"]) == (st2["n_newton"], st2["n_mv"])
    assert np.abs(v3[:2] - np.stack([lift(v2[0]), lift(v2[1])])).max() < 1e-9 * np.abs(v2).max()
    assert np.abs(v3[2]).max() < 1e-12


def test_solve_3d_converges_divergence_free():
    P, _, _ = _problem3d(4)
    v, st = R.solve(P, tol=1e-2)
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2 and st["J"] < st["J0"]
    assert np.abs(R.div(v)).max() < 1e-10 * max(np.abs(v).max(), 1e-30)


def test_gauss_newton_matvec_is_the_derivative_of_the_gradient_at_zero_residual():
    """With m_R := m(1) for the linearization point (lam = 0), the Gauss-Newton Hessian is the
    full Hessian, so H v~ matches central differences of g along v~ up to the O(h_t^2) of
    optimize-then-discretize derivatives: the mismatch falls by ~4 per halving of h_t."""
    errs = []
    for nt in (2, 4, 8):
        P, v, d = _problem3d(nt, 0.0)
        m, _ = R.state_solve(P.mT, v, nt)
        P = R.Registration3D(P.mT, m[-1], nt, P.beta_v, 0.0)
        eps = 1e-4
        fd = (P.gradient(v + eps * d)[0] - P.gradient(v - eps * d)[0]) / (2 * eps)
        P.gradient(v)
        H = P.matvec(d)
        errs.append(np.linalg.norm(fd - H) / np.linalg.norm(fd))
    assert errs[-1] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0
