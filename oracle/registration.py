"""Reduced-space (Gauss-)Newton-Krylov registration (oracle; test
infrastructure only).

Follows, in the paper's order and notation:
  * objective J[v] (Eq. (e:objective)) with the mass source eliminated
    through w = div v (Eq. (e:constraint-divv));
  * reduced gradient g = beta_v A[v] + K[b] (Eq. (e:control-eq-elim)), with
    the state solve, adjoint solve and body force of Algorithm 1;
  * Gauss-Newton Hessian matvec H v~ = beta_v B[v~] + L[b~]
    (Eq. (e:inc-control-eq-elim)) with the lambda terms dropped (Sec. 4), or the
    full Newton matvec that keeps them (hessian="full");
  * PCG inner iteration, Algorithm 2, preconditioned by (beta_v A)^-1
    (Appendix E);
  * Armijo backtracking line search (Sec. 4: Nocedal-Wright Algorithm 3.1,
    default parameters) and the Newton outer iteration, Algorithm 1.

Readings of passages the paper leaves open or garbles:
  * PCG stop test: Algorithm 2 prints "||r_{l+1}||_2 < eta_k"; the forcing
    sequence is stated to be relative to the gradient (Appendix E text,
    Dembo/Eisenstat), so the test is ||r_{l+1}|| < eta_k ||g_k||.  The loop
    bound "l < n" is capped at ``maxit_pcg`` (default 100).
  * Forcing term eta_k = min(0.5, sqrt(||g_k|| / ||g_0||)) (Algorithm 2), with
    g_0 the gradient at the initial iterate v_0 of Algorithm 1 (for a warm
    start, the gradient at the warm start).
  * Armijo constants: alpha_0 = 1, rho = 1/2, c1 = 1e-4, at most 20
    backtracks.  Acceptance J(v + alpha v~) <= J(v) + c1 alpha <g, v~>.
  * Outer stop: ||g_k|| / ||g_ref|| <= tol (unsquared, quadrature-weighted L2);
    g_ref is the gradient at v = 0 (equal to g_0 for a zero start).  The
    paper's table reports the squared ratio; both are returned.
  * Norms and inner products are the trapezoidal-rule L2 ones; all the
    ratios above are invariant to that choice of scaling.
  * Objective term for 0 < beta_w < inf: (beta_w / 2) <(-Lap + I) w, w> with
    w = div v (Eq. (e:reg-w)).
  * If PCG meets a non-positive curvature <s, H s> <= 0 it stops (a plain
    safeguard; the Gauss-Newton Hessian is positive definite in exact
    arithmetic, Sec. 4; the full Hessian need not be far from a minimizer, and
    this guard is then what keeps the step a descent direction).  If the returned step is not a descent direction
    (<g, v~> >= 0) the preconditioned steepest-descent step -(beta_v A)^-1 g
    is used instead.
  * nt policy: "fixed" uses nt as given; "cfl" uses, at every outer
    iteration, nt_used = max(nt, ceil(max|v| n / (2 pi c_max))) with
    c_max = 0.25 and n = max(n1, n2) (Sec. 5.1 adapts nt to the CFL
    condition).
"""
import math

import numpy as np

from . import shear as shear_ops
from .spectral import (H1, H2, H3, apply_A, apply_K, apply_precond, apply_W, div,
                       inner, norm)
from .transport import (adjoint_solve, body_force, grad_history,
                        inc_adjoint_solve_full, inc_state_solve, state_solve)

STATUS_OK = 0
STATUS_LINESEARCH = 5
STATUS_MAXIT = 10


class Registration:
    """One registration problem: template m_T, reference m_R (both (n1, n2)),
    nt time steps, regularization norm (1 = H1, 2 = H2, 3 = H3), beta_v, beta_w
    (0: gamma = 0; inf: incompressible; else mass source weight) and shear
    knob s (0 = quadratic model; s != 0 requires H1)."""

    def __init__(self, mT, mR, nt, regnorm=H1, beta_v=1e-2, beta_w=np.inf, shear=0.0, hessian="gn"):
        self.mT = np.asarray(mT, dtype=np.float64)
        self.mR = np.asarray(mR, dtype=np.float64)
        self.nt = int(nt)
        self.regnorm = int(regnorm)
        self.beta_v = float(beta_v)
        self.beta_w = float(beta_w)
        self.shear = float(shear)
        if hessian not in ("gn", "full"):
            raise ValueError("hessian must be 'gn' (Gauss-Newton) or 'full'")
        self.hessian = hessian
        if self.shear != 0.0:
            if self.regnorm != H1:
                raise ValueError("shear control requires H1")
            self.nu = shear_ops.nu_from_shear(self.shear)
        self.v = None
        self.n_pde = 0

    # ---- regularization pieces -------------------------------------------
    def reg_energy(self, v):
        e = 0.0
        if self.shear != 0.0:
            e = shear_ops.energy(v, self.nu, self.beta_v)
        else:
            e = 0.5 * self.beta_v * inner(apply_A(v, self.regnorm), v)
        if 0.0 < self.beta_w < np.inf:
            w = div(v)
            e += 0.5 * self.beta_w * inner(apply_W(w), w)
        return e

    def precond(self, r):
        regnorm = H1 if self.shear != 0.0 else self.regnorm
        return apply_precond(r, regnorm, self.beta_v)

    # ---- objective, gradient, Hessian ------------------------------------
    def objective(self, v, nt=None):
        """J[v] (Eq. (e:objective)); one forward state solve."""
        nt = self.nt if nt is None else nt
        m = state_solve(self.mT, v, nt)
        self.n_pde += 1
        r = self.mR - m[-1]
        return 0.5 * inner(r, r) + self.reg_energy(v), m

    def gradient(self, v, nt=None):
        """Reduced gradient (Eq. (e:control-eq-elim)); also fixes the
        linearization point used by ``matvec``.  Returns (g, J)."""
        v = np.asarray(v, dtype=np.float64)
        nt = self.nt if nt is None else nt
        J, m = self.objective(v, nt)
        lam = adjoint_solve(self.mR - m[-1], v, nt)
        self.n_pde += 1
        gm = grad_history(m)
        b = body_force(lam, gm)
        if self.shear != 0.0 and np.isinf(self.beta_w):
            g = shear_ops.leray(self.beta_v * shear_ops.first_variation(v, self.nu) + b)
        elif self.shear != 0.0 and self.beta_w > 0.0:
            g = shear_ops.reduced_gradient_mass(v, b, self.nu, self.beta_v, self.beta_w)
        elif self.shear != 0.0:
            g = self.beta_v * shear_ops.first_variation(v, self.nu) + b
        else:
            g = self.beta_v * apply_A(v, self.regnorm) + apply_K(b, self.regnorm, self.beta_v, self.beta_w)
        self.v, self.m, self.gradm, self.lam, self.b, self.nt_lin = v, m, gm, lam, b, nt
        return g, J

    def matvec(self, vt):
        """Hessian matvec H v~ (Eqs. (e:inc-state-eq-elim), (e:inc-adj-eq-elim),
        (e:inc-control-eq-elim)) at the point of the last ``gradient`` call (Algorithm 2):
        Gauss-Newton (lambda terms dropped, Sec. 4) unless ``self.hessian == "full"``, which
        keeps them: the source -div(lam v~) of the incremental adjoint and the term
        lam grad m~ of the incremental body force b~ = int lam~ grad m + lam grad m~ dt."""
        vt = np.asarray(vt, dtype=np.float64)
        nt = self.nt_lin
        mt = inc_state_solve(self.v, vt, self.gradm, nt)
        self.n_pde += 2
        if self.hessian == "full":
            lt = inc_adjoint_solve_full(-mt[-1], self.v, vt, self.lam, nt)
            bt = body_force(lt, self.gradm) + body_force(self.lam, grad_history(mt))
        else:
            lt = adjoint_solve(-mt[-1], self.v, nt)
            bt = body_force(lt, self.gradm)
        self.bt = bt
        if self.shear != 0.0 and np.isinf(self.beta_w):
            return shear_ops.leray(self.beta_v * shear_ops.second_variation(self.v, vt, self.nu) + bt)
        if self.shear != 0.0 and self.beta_w > 0.0:
            return shear_ops.hessian_mass(self.v, vt, bt, self.nu, self.beta_v, self.beta_w)
        if self.shear != 0.0:
            return self.beta_v * shear_ops.second_variation(self.v, vt, self.nu) + bt
        return self.beta_v * apply_A(vt, self.regnorm) + apply_K(bt, self.regnorm, self.beta_v, self.beta_w)

    # ---- Algorithm 2 -----------------------------------------------------
    def pcg(self, g, eta, maxit):
        """Returns (v~, iterations, ||r|| / ||g||, hit_maxit)."""
        vt = np.zeros_like(g)
        r = -g
        z = self.precond(r)
        s = z.copy()
        rz = inner(r, z)
        gnorm = norm(g)
        it = 0
        hit_max = True
        for _ in range(maxit):
            Hs = self.matvec(s)
            it += 1
            sHs = inner(s, Hs)
            if sHs <= 0.0:
                hit_max = False
                if it == 1:
                    vt = s.copy()
                break
            kappa = rz / sHs
            vt = vt + kappa * s
            r = r - kappa * Hs
            if norm(r) < eta * gnorm:
                hit_max = False
                break
            z = self.precond(r)
            rz_new = inner(z, r)
            mu = rz_new / rz
            s = z + mu * s
            rz = rz_new
        return vt, it, norm(r) / gnorm, hit_max

    # ---- Algorithm 1 -----------------------------------------------------
    def nt_for(self, v, policy, c_max=0.25):
        if policy == "fixed":
            return self.nt
        n = max(self.mT.shape)
        vmax = float(np.max(np.sqrt(v[0] ** 2 + v[1] ** 2)))
        return max(self.nt, int(math.ceil(vmax * n / (2.0 * math.pi * c_max))))

    def solve(self, v0=None, tol=1e-2, maxit_newton=50, maxit_pcg=100,
              c1=1e-4, rho=0.5, max_ls=20, nt_policy="fixed"):
        """Globalized inexact Gauss-Newton-Krylov solve (Algorithm 1).
        Returns (v, stats dict)."""
        n1, n2 = self.mT.shape
        zero = np.zeros((2, n1, n2))
        self.n_pde = 0
        stats = dict(n_newton=0, n_mv=0, n_ls=0, n_pcg_maxit=0, status=STATUS_OK)
        v = zero if v0 is None else np.asarray(v0, dtype=np.float64).copy()
        nt = self.nt_for(v, nt_policy)
        if v0 is not None:
            g_ref, _ = self.gradient(zero, self.nt)
            gref = norm(g_ref)
        g, J = self.gradient(v, nt)
        if v0 is None:
            gref = norm(g)
        gnorm = norm(g)
        gstart = gnorm
        stats["J0"] = J
        k = 0
        while True:
            if gref == 0.0 or gnorm / gref <= tol:
                break
            if k >= maxit_newton:
                stats["status"] = STATUS_MAXIT
                break
            eta = min(0.5, math.sqrt(gnorm / gstart))
            vt, it, relres, hit = self.pcg(g, eta, maxit_pcg)
            stats["n_mv"] += it
            stats["n_pcg_maxit"] += int(hit)
            gv = inner(g, vt)
            if gv >= 0.0:
                vt = -self.precond(g)
                gv = inner(g, vt)
            alpha = 1.0
            accepted = False
            for _ in range(max_ls):
                Jt, _ = self.objective(v + alpha * vt, nt)
                stats["n_ls"] += 1
                if Jt <= J + c1 * alpha * gv:
                    accepted = True
                    break
                alpha *= rho
            if not accepted:
                stats["status"] = STATUS_LINESEARCH
                break
            v = v + alpha * vt
            k += 1
            nt = self.nt_for(v, nt_policy)
            g, J = self.gradient(v, nt)
            gnorm = norm(g)
        stats["n_newton"] = k
        stats["n_pde"] = self.n_pde
        stats["J"] = J
        stats["gnorm_rel"] = gnorm / gref if gref > 0 else 0.0
        stats["gnorm_rel_sq"] = stats["gnorm_rel"] ** 2
        r1 = self.mR - self.m[-1]
        r0 = self.mR - self.mT
        stats["rnorm_rel_sq"] = inner(r1, r1) / inner(r0, r0) if inner(r0, r0) > 0 else 0.0
        stats["nt_used"] = nt
        return v, stats
