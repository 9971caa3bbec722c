"""Three-dimensional registration operators (oracle; test infrastructure only).

The paper states its method for d = 2 and names the three-dimensional case as the next step
(Conclusions); the equations of Sec. 3 are written for a general dimension d, so this module takes
them over unchanged for d = 3 on the periodic box [0, 2 pi)^3 with the H1 seminorm:

  * state, Eq. (e:state-eq-elim): d_t m + grad m . v = 0, m(0) = m_T;
  * adjoint, Eq. (e:adj-eq-elim): -d_t lam - div(lam v) = 0, lam(1) = m_R - m(1);
  * body force b = int_0^1 lam grad m dt and reduced gradient g = beta_v A v + K b,
    Eq. (e:control-eq-elim), with A = -Lap (symbol |k|^2) and the projection K of
    Eq. (e:project-body-force), K^ = I - k~ k~^T / (|k~|^2 + beta_v |k|^2 / (beta_w (1 + |k|^2)))
    (the symbol of A over that of the inverse Laplacian of the elimination; K^ = I - k~ k~^T /
    |k~|^2 for beta_w = inf, K = I for beta_w = 0);
  * Gauss-Newton matvec, Eqs. (e:inc-state-eq-elim), (e:inc-adj-eq-elim),
    (e:inc-control-eq-elim): d_t m~ + grad m~ . v + grad m . v~ = 0, m~(0) = 0;
    lam~(1) = -m~(1) with the adjoint's transport; H v~ = beta_v A v~ + K b~,
    b~ = int lam~ grad m dt;
  * objective J = 1/2 ||m_R - m(1)||^2 + beta_v / 2 <A v, v>, plus beta_w / 2 <(-Lap + I) w, w>
    with w = div v when 0 < beta_w < inf (Eq. (e:reg-w)).

Readings shared with the two-dimensional oracle: Heun's method for the RK2 steps (sources of
the incremental state at t_j and t_{j+1}), trapezoidal weights in time, odd symbols k~ with
the Nyquist entry set to zero for grad and div, the full even symbol |k|^2 for A and M^,
the trapezoidal inner product h1 h2 h3 sum.  The own radix-2 FFT of ``oracle.fft`` runs along
each of the three axes.
"""
import math

import numpy as np

from .fft import fft


def fftn3(x):
    return fft(fft(fft(x, axis=-3), axis=-2), axis=-1)


def ifftn3(X):
    n = X.shape[-3] * X.shape[-2] * X.shape[-1]
    return fft(fft(fft(X, axis=-3, inverse=True), axis=-2, inverse=True), axis=-1, inverse=True) / n


def _wavenumbers(n):
    k = np.concatenate([np.arange(0, n // 2), np.arange(-n // 2, 0)]).astype(np.float64)
    k_odd = k.copy()
    k_odd[n // 2] = 0.0
    k_even = k.copy()
    k_even[n // 2] = n / 2.0
    return k_odd, k_even


def symbols(shape):
    """(k~1, k~2, k~3, |k|^2) on the full n1 x n2 x n3 spectrum."""
    o1, e1 = _wavenumbers(shape[0])
    o2, e2 = _wavenumbers(shape[1])
    o3, e3 = _wavenumbers(shape[2])
    K1, K2, K3 = np.meshgrid(o1, o2, o3, indexing="ij")
    E1, E2, E3 = np.meshgrid(e1, e2, e3, indexing="ij")
    return K1, K2, K3, E1 ** 2 + E2 ** 2 + E3 ** 2


def grid_coords(shape):
    xs = [2.0 * np.pi * np.arange(n) / n for n in shape]
    return np.meshgrid(*xs, indexing="ij")


def inner(f, g):
    """Trapezoidal L2 inner product h1 h2 h3 sum f g over every component."""
    n1, n2, n3 = np.shape(f)[-3:]
    h = (2.0 * np.pi) ** 3 / (n1 * n2 * n3)
    return float(h * np.sum(np.asarray(f, dtype=np.float64) * np.asarray(g, dtype=np.float64)))


def norm(f):
    return float(np.sqrt(inner(f, f)))


def grad(f):
    K1, K2, K3, _ = symbols(f.shape)
    F = fftn3(f)
    return np.stack([np.real(ifftn3(1j * K * F)) for K in (K1, K2, K3)])


def div(u):
    K1, K2, K3, _ = symbols(u.shape[-3:])
    return np.real(ifftn3(1j * (K1 * fftn3(u[0]) + K2 * fftn3(u[1]) + K3 * fftn3(u[2]))))


def apply_A(v):
    """A v = -Lap v per component (symbol |k|^2, the H1 seminorm's first variation)."""
    _, _, _, KK = symbols(v.shape[-3:])
    return np.stack([np.real(ifftn3(KK * fftn3(v[c]))) for c in range(3)])


def apply_K(b, beta_v, beta_w):
    """K b of Eq. (e:project-body-force) for the H1 seminorm in three dimensions."""
    if beta_w == 0.0:
        return np.array(b, dtype=np.float64, copy=True)
    K1, K2, K3, KK = symbols(b.shape[-3:])
    kk = K1 ** 2 + K2 ** 2 + K3 ** 2
    denom = kk if np.isinf(beta_w) else kk + beta_v * KK / (beta_w * (1.0 + KK))
    coef = np.zeros_like(kk)
    nz = kk > 0.0
    coef[nz] = 1.0 / denom[nz]
    B = [fftn3(b[c]) for c in range(3)]
    kb = K1 * B[0] + K2 * B[1] + K3 * B[2]
    return np.stack([np.real(ifftn3(B[c] - coef * K * kb)) for c, K in enumerate((K1, K2, K3))])


def trapezoid_weights(nt):
    w = np.full(nt + 1, 1.0 / nt)
    w[0] *= 0.5
    w[-1] *= 0.5
    return w


def _dot(gf, v):
    return gf[0] * v[0] + gf[1] * v[1] + gf[2] * v[2]


def state_solve(mT, v, nt):
    """History m[j] = m(t_j), j = 0..nt, and the gradient history grad m[j]."""
    h = 1.0 / nt
    m = np.empty((nt + 1,) + mT.shape)
    m[0] = mT
    for j in range(nt):
        k1 = -_dot(grad(m[j]), v)
        ms = m[j] + h * k1
        k2 = -_dot(grad(ms), v)
        m[j + 1] = m[j] + 0.5 * h * (k1 + k2)
    gm = np.stack([grad(m[j]) for j in range(nt + 1)])
    return m, gm


def adjoint_solve(lam_final, v, nt):
    """lam[j] = lam(t_j) backward from lam(1): with tau = 1 - t, d_tau lam = div(lam v)."""
    h = 1.0 / nt
    lam = np.empty((nt + 1,) + lam_final.shape)
    lam[nt] = lam_final
    for j in range(nt, 0, -1):
        k1 = div(lam[j] * v)
        ls = lam[j] + h * k1
        k2 = div(ls * v)
        lam[j - 1] = lam[j] + 0.5 * h * (k1 + k2)
    return lam


def body_force(lam, gm):
    w = trapezoid_weights(lam.shape[0] - 1)
    return sum(w[j] * lam[j] * gm[j] for j in range(lam.shape[0]))


def inc_state_solve(v, vt, gm, nt):
    h = 1.0 / nt
    mt = np.zeros((nt + 1,) + v.shape[1:])
    for j in range(nt):
        k1 = -_dot(grad(mt[j]), v) - _dot(gm[j], vt)
        ms = mt[j] + h * k1
        k2 = -_dot(grad(ms), v) - _dot(gm[j + 1], vt)
        mt[j + 1] = mt[j] + 0.5 * h * (k1 + k2)
    return mt


class Registration3D:
    """Objective, reduced gradient and Gauss-Newton matvec of one 3-D registration problem."""

    def __init__(self, mT, mR, nt, beta_v, beta_w=np.inf):
        self.mT = np.asarray(mT, dtype=np.float64)
        self.mR = np.asarray(mR, dtype=np.float64)
        self.nt, self.beta_v, self.beta_w = nt, beta_v, beta_w

    def objective(self, v):
        m, gm = state_solve(self.mT, v, self.nt)
        r = self.mR - m[-1]
        J = 0.5 * inner(r, r) + 0.5 * self.beta_v * inner(apply_A(v), v)
        if 0.0 < self.beta_w < np.inf:
            w = div(v)
            _, _, _, KK = symbols(w.shape)
            J += 0.5 * self.beta_w * inner(np.real(ifftn3((1.0 + KK) * fftn3(w))), w)
        return J, m, gm

    def gradient(self, v):
        """(g, J); fixes the linearization point of ``matvec``."""
        v = np.asarray(v, dtype=np.float64)
        J, m, gm = self.objective(v)
        lam = adjoint_solve(self.mR - m[-1], v, self.nt)
        b = body_force(lam, gm)
        self.v, self.gm, self.b = v, gm, b
        return self.beta_v * apply_A(v) + apply_K(b, self.beta_v, self.beta_w), J

    def matvec(self, vt):
        vt = np.asarray(vt, dtype=np.float64)
        mt = inc_state_solve(self.v, vt, self.gm, self.nt)
        lt = adjoint_solve(-mt[-1], self.v, self.nt)
        bt = body_force(lt, self.gm)
        self.bt = bt
        return self.beta_v * apply_A(vt) + apply_K(bt, self.beta_v, self.beta_w)


def apply_precond(r, beta_v):
    """(beta_v A)^-1 r with the k = 0 symbol of A replaced by 1 (App. E, as in 2-D)."""
    _, _, _, KK = symbols(r.shape[-3:])
    sym = beta_v * np.where(KK > 0.0, KK, 1.0)
    return np.stack([np.real(ifftn3(fftn3(r[c]) / sym)) for c in range(3)])


def _pcg(P, g, eta, maxit):
    """Algorithm 2 with the spectral preconditioner: (v~, iterations)."""
    vt = np.zeros_like(g)
    r = -g
    z = apply_precond(r, P.beta_v)
    s = z.copy()
    rz = inner(r, z)
    gnorm = norm(g)
    it = 0
    for _ in range(maxit):
        Hs = P.matvec(s)
        it += 1
        sHs = inner(s, Hs)
        if sHs <= 0.0:
            if it == 1:
                vt = s.copy()
            break
        kappa = rz / sHs
        vt = vt + kappa * s
        r = r - kappa * Hs
        if norm(r) < eta * gnorm:
            break
        z = apply_precond(r, P.beta_v)
        rz_new = inner(z, r)
        s = z + (rz_new / rz) * s
        rz = rz_new
    return vt, it


def solve(P, tol=1e-2, maxit_newton=50, maxit_pcg=100, c1=1e-4, rho=0.5, max_ls=20):
    """Algorithm 1 from v = 0 (inexact Gauss-Newton-Krylov with Armijo backtracking, forcing
    eta_k = min(0.5, sqrt(||g_k|| / ||g_0||)), stop at ||g|| <= tol ||g_0||), the same steps as
    the two-dimensional oracle's solve.  Returns (v, stats)."""
    v = np.zeros((3,) + P.mT.shape)
    g, J = P.gradient(v)
    g0 = gnorm = norm(g)
    stats = dict(n_newton=0, n_mv=0, n_ls=0, status=0, J0=J)
    while g0 > 0.0 and gnorm / g0 > tol:
        if stats["n_newton"] >= maxit_newton:
            stats["status"] = 10
            break
        vt, it = _pcg(P, g, min(0.5, math.sqrt(gnorm / g0)), maxit_pcg)
        stats["n_mv"] += it
        gv = inner(g, vt)
        if gv >= 0.0:
            vt = -apply_precond(g, P.beta_v)
            gv = inner(g, vt)
        alpha, accepted = 1.0, False
        for _ in range(max_ls):
            stats["n_ls"] += 1
            if P.objective(v + alpha * vt)[0] <= J + c1 * alpha * gv:
                accepted = True
                break
            alpha *= rho
        if not accepted:
            stats["status"] = 5
            break
        v = v + alpha * vt
        stats["n_newton"] += 1
        g, J = P.gradient(v)
        gnorm = norm(g)
    stats.update(J=J, gnorm_rel=gnorm / g0 if g0 > 0 else 0.0)
    return v, stats
