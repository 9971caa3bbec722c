"""Hyperbolic transport solves in pseudo-time t in [0, 1] (oracle; test
infrastructure only).

Time integration: the paper uses "an explicit second order Runge-Kutta
method" (Sec. 4) without naming the variant.  The oracle uses Heun's method
(explicit trapezoid):  y* = y_j + h f(t_j, y_j),  y_{j+1} = y_j + h/2 (f(t_j, y_j)
+ f(t_{j+1}, y*)), h = 1/nt.  For a stationary velocity every two-stage RK2
gives the same update for the homogeneous equations; the variant only matters
for the source term of the incremental state equation, which is evaluated at
t_j and t_{j+1} from the stored state history.

Time quadrature: trapezoidal rule (Sec. 4), weights h (1/2, 1, ..., 1, 1/2).
"""
import numpy as np

from .spectral import grad, div


def trapezoid_weights(nt):
    w = np.full(nt + 1, 1.0 / nt)
    w[0] *= 0.5
    w[-1] *= 0.5
    return w


def advect(f, v):
    """grad f . v (pointwise product of the spectral gradient with v)."""
    g = grad(f)
    return g[0] * v[0] + g[1] * v[1]


def state_solve(mT, v, nt):
    """State equation, Eq. (e:state-eq-elim): d_t m + grad m . v = 0, m(0) = m_T.
    Returns the history m[j] = m(t_j), j = 0..nt (Algorithm 1, forward solve)."""
    h = 1.0 / nt
    m = np.empty((nt + 1,) + mT.shape)
    m[0] = mT
    for j in range(nt):
        k1 = -advect(m[j], v)
        ms = m[j] + h * k1
        k2 = -advect(ms, v)
        m[j + 1] = m[j] + 0.5 * h * (k1 + k2)
    return m


def adjoint_solve(lam_final, v, nt):
    """Adjoint equation, Eq. (e:adj-eq-elim): -d_t lam - div(lam v) = 0, solved
    backward in time from lam(1) = lam_final.  With tau = 1 - t this is
    d_tau lam = div(lam v).  Returns lam[j] = lam(t_j), j = 0..nt.  The same
    routine solves the Gauss-Newton incremental adjoint equation
    (Eq. (e:inc-adj-eq-elim) with the lambda term dropped, Sec. 4)."""
    h = 1.0 / nt
    lam = np.empty((nt + 1,) + lam_final.shape)
    lam[nt] = lam_final
    for j in range(nt, 0, -1):
        k1 = div(lam[j] * v)
        ls = lam[j] + h * k1
        k2 = div(ls * v)
        lam[j - 1] = lam[j] + 0.5 * h * (k1 + k2)
    return lam


def body_force(lam, gradm):
    """b = int_0^1 lam grad m dt (Sec. 3.1), trapezoidal rule in time.
    lam: (nt+1, n1, n2); gradm: (nt+1, 2, n1, n2)."""
    nt = lam.shape[0] - 1
    w = trapezoid_weights(nt)
    b = np.zeros(gradm.shape[1:])
    for j in range(nt + 1):
        b += w[j] * lam[j] * gradm[j]
    return b


def inc_state_solve(v, vt, gradm, nt):
    """Incremental state equation, Eq. (e:inc-state-eq-elim):
    d_t m~ + grad m~ . v + grad m . v~ = 0, m~(0) = 0.  gradm holds grad m(t_j)
    for j = 0..nt.  Returns the history m~[j]."""
    h = 1.0 / nt
    mt = np.zeros((nt + 1,) + v.shape[1:])
    for j in range(nt):
        src0 = -(gradm[j, 0] * vt[0] + gradm[j, 1] * vt[1])
        src1 = -(gradm[j + 1, 0] * vt[0] + gradm[j + 1, 1] * vt[1])
        k1 = -advect(mt[j], v) + src0
        ms = mt[j] + h * k1
        k2 = -advect(ms, v) + src1
        mt[j + 1] = mt[j] + 0.5 * h * (k1 + k2)
    return mt


def inc_adjoint_solve_full(lam_final, v, vt, lam, nt):
    """Incremental adjoint of the full Newton step, Eq. (e:inc-adj-eq-elim) with the lambda
    term kept: -d_t lam~ - div(lam~ v) - div(lam v~) = 0, solved backward from
    lam~(1) = lam_final.  With tau = 1 - t: d_tau lam~ = div(lam~ v) + div(lam v~); the source
    div(lam v~) is evaluated from the adjoint history lam[j] at the stage times t_j and
    t_{j-1} (Heun, as for the incremental state).  Returns lam~[j], j = 0..nt."""
    h = 1.0 / nt
    lt = np.empty((nt + 1,) + lam_final.shape)
    lt[nt] = lam_final
    for j in range(nt, 0, -1):
        k1 = div(lt[j] * v) + div(lam[j] * vt)
        ls = lt[j] + h * k1
        k2 = div(ls * v) + div(lam[j - 1] * vt)
        lt[j - 1] = lt[j] + 0.5 * h * (k1 + k2)
    return lt


def grad_history(m):
    return np.stack([grad(m[j]) for j in range(m.shape[0])])


def displacement_solve(v, nt):
    """Displacement field, Eq. (e:displacement): d_t u + (grad u) v = v, u(0) = 0, i.e. per
    component c the transport d_t u_c + grad u_c . v = v_c with a source constant in time
    (Heun, as for the state equation).  Returns u_1 = u(t = 1) as (2, n1, n2); the
    deformation map (Eulerian, where points originate from) is y = x - u_1."""
    h = 1.0 / nt
    u = np.zeros_like(np.asarray(v, dtype=np.float64))
    for c in range(2):
        uc = np.zeros(v.shape[1:])
        for _ in range(nt):
            k1 = -advect(uc, v) + v[c]
            us = uc + h * k1
            k2 = -advect(us, v) + v[c]
            uc = uc + 0.5 * h * (k1 + k2)
        u[c] = uc
    return u


def defgrad_solve(v, nt):
    """Deformation gradient, Eq. (e:def-grad): d_t F + (v . grad) F = (grad v) F,
    F(0) = I, with (grad v)_{ac} = d_c v_a.  Returns F1 = F(t=1) as (2, 2, n1, n2)."""
    h = 1.0 / nt
    n1, n2 = v.shape[-2:]
    gv = np.stack([grad(v[0]), grad(v[1])])  # gv[a, c] = d_c v_a

    def rhs(F):
        out = np.empty_like(F)
        for a in range(2):
            for b in range(2):
                out[a, b] = -advect(F[a, b], v) + gv[a, 0] * F[0, b] + gv[a, 1] * F[1, b]
        return out

    F = np.zeros((2, 2, n1, n2))
    F[0, 0] = 1.0
    F[1, 1] = 1.0
    for _ in range(nt):
        k1 = rhs(F)
        Fs = F + h * k1
        k2 = rhs(Fs)
        F = F + 0.5 * h * (k1 + k2)
    return F


def defgrad_measures(F1):
    """det F1 and D = ||F1 - I||_F pointwise (Appendix F, performance measures)."""
    det = F1[0, 0] * F1[1, 1] - F1[0, 1] * F1[1, 0]
    D = np.sqrt((F1[0, 0] - 1.0) ** 2 + F1[0, 1] ** 2 + F1[1, 0] ** 2 + (F1[1, 1] - 1.0) ** 2)
    return det, D
