"""Pins for the oracle's full-Newton Hessian and the H3 seminorm (CPU only).

Full Newton keeps the lambda terms the Gauss-Newton approximation drops (Sec. 4): the source
-div(lam v~) of the incremental adjoint (Eq. (e:inc-adj-eq-elim)) and lam grad m~ in the
incremental body force.  With them the matvec is the derivative of the reduced gradient, so
central differences of g along v~ must match H v~ at ANY linearization point, up to the
O(h_t^2) consistency of optimize-then-discretize derivatives (observed order 2); the
Gauss-Newton matvec must not (its mismatch is O(lam), not O(h_t^2)).  Dropping either lambda
term, or flipping a sign, breaks the order-2 convergence.  At a zero-residual point (lam = 0)
the two matvecs coincide exactly.

H3 (App. A.1: "the same arguments hold", the triharmonic control equation): symbol |k|^6 on
single Fourier modes, the mass-source projection's eigenvalue along k, and the gradient
against finite differences of J (order 2)."""
import math

import numpy as np
import pytest

from oracle import spectral as S
from oracle import transport as T
from oracle.registration import Registration
from paper_1503_00757_gb300 import synth


def _fd_gradient(P, v, d, eps):
    gp, _ = P.gradient(v + eps * d)
    gm, _ = P.gradient(v - eps * d)
    return (gp - gm) / (2 * eps)


def _mismatch(hessian, nt, regnorm=S.H1, beta_w=math.inf):
    mT, mR, vs = synth.blobs_pair(32, 1000, vmax=0.4, kmax=3)
    P = Registration(mT, mR, nt, regnorm=regnorm, beta_v=1e-2, beta_w=beta_w, hessian=hessian)
    v = 0.5 * vs
    d = synth.velocity(32, 32, 4, 0.3, np.random.default_rng(1))
    fd = _fd_gradient(P, v, d, 1e-4)
    P.gradient(v)
    H = P.matvec(d)
    return np.linalg.norm(fd - H) / np.linalg.norm(fd)


@pytest.mark.parametrize("beta_w", [math.inf, 0.0])
def test_full_hessian_is_the_derivative_of_the_gradient(beta_w):
    errs = [_mismatch("full", nt, beta_w=beta_w) for nt in (4, 8, 16)]
    assert errs[-1] < 2e-4
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0
    gn = _mismatch("gn", 16, beta_w=beta_w)
    assert gn > 50 * errs[-1]  # the lambda terms matter at a nonzero residual


def test_full_equals_gauss_newton_at_zero_residual():
    mT, _, vs = synth.blobs_pair(32, 1001, vmax=0.4, kmax=3)
    v = 0.5 * vs
    nt = 8
    mR = T.state_solve(mT, v, nt)[-1]  # m_R := m_1(v): lam = m_R - m_1 = 0
    d = synth.velocity(32, 32, 4, 0.3, np.random.default_rng(2))
    out = []
    for hs in ("gn", "full"):
        P = Registration(mT, mR, nt, regnorm=S.H1, beta_v=1e-2, hessian=hs)
        P.gradient(v)
        assert np.abs(P.lam).max() == 0.0
        out.append(P.matvec(d))
    assert np.array_equal(out[0], out[1])


def test_full_hessian_symmetry_order_two():
    """<H u, w> = <u, H w> up to the O(h_t^2) of the time discretization (H is the Hessian
    of J for gamma = 0, a symmetric operator)."""
    mT, mR, vs = synth.blobs_pair(32, 1000, vmax=0.4, kmax=3)
    u = synth.velocity(32, 32, 4, 0.3, np.random.default_rng(3), grad_fraction=0.5)
    w = synth.velocity(32, 32, 4, 0.3, np.random.default_rng(4), grad_fraction=0.5)
    errs = []
    for nt in (4, 8, 16):
        P = Registration(mT, mR, nt, regnorm=S.H1, beta_v=1e-2, beta_w=0.0, hessian="full")
        P.gradient(0.5 * vs)
        a, b = S.inner(P.matvec(u), w), S.inner(u, P.matvec(w))
        errs.append(abs(a - b) / max(abs(a), abs(b)))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_full_newton_solve_converges():
    mT, mR, _ = synth.blobs_pair(32, 1000)
    stats = {}
    for hs in ("gn", "full"):
        P = Registration(mT, mR, 8, regnorm=S.H1, beta_v=1e-2, hessian=hs)
        v, st = P.solve(tol=1e-3)
        assert st["status"] == 0 and st["gnorm_rel"] <= 1e-3 and st["J"] < st["J0"]
        assert np.abs(S.div(v)).max() < 1e-10
        stats[hs] = (st, v)
    # same minimizer
    vg, vf = stats["gn"][1], stats["full"][1]
    assert np.linalg.norm(vg - vf) / np.linalg.norm(vg) < 2e-2


def test_h3_symbol_on_single_modes():
    n = 32
    X1, X2 = S.grid_coords(n, n)
    for k1, k2 in [(1, 0), (2, 3), (5, -4)]:
        f = np.cos(k1 * X1 + k2 * X2)
        v = np.stack([f, 0.5 * f])
        kk = k1 * k1 + k2 * k2
        assert np.abs(S.apply_A(v, S.H3) - kk ** 3 * v).max() < 1e-8 * kk ** 3


def test_h3_mass_source_projection_eigenvalue():
    """K applied to a gradient field along k scales it by beta_v |k|^4 / (beta_w (1 + |k|^2)
    + beta_v |k|^4) for A = |k|^6 (the eigenvalue 1 - 1/M^ of Eq. (e:project-body-force) with
    the H3 symbol); fields orthogonal to k are kept."""
    n, bv, bw = 32, 1e-3, 1e-2
    X1, X2 = S.grid_coords(n, n)
    for k1, k2 in [(1, 1), (3, -2)]:
        s = np.sin(k1 * X1 + k2 * X2)
        grad_mode = np.stack([k1 * s, k2 * s])
        perp_mode = np.stack([-k2 * s, k1 * s])
        kk = k1 * k1 + k2 * k2
        lam = bv * kk ** 2 / (bw * (1 + kk) + bv * kk ** 2)
        assert np.abs(S.apply_K(grad_mode, S.H3, bv, bw) - lam * grad_mode).max() < 1e-12
        assert np.abs(S.apply_K(perp_mode, S.H3, bv, bw) - perp_mode).max() < 1e-12


def test_h3_gradient_matches_fd_second_order():
    errs = []
    for nt in (4, 8, 16):
        mT, mR, vs = synth.blobs_pair(32, 1000)
        P = Registration(mT, mR, nt, regnorm=S.H3, beta_v=1e-5, beta_w=0.0)
        v = 0.5 * vs
        d = synth.velocity(32, 32, 6, 0.2, np.random.default_rng(1), grad_fraction=1.0)
        g, _ = P.gradient(v)
        eps = 1e-4
        fd = (P.objective(v + eps * d)[0] - P.objective(v - eps * d)[0]) / (2 * eps)
        errs.append(abs(S.inner(g, d) - fd) / abs(fd))
    assert errs[-1] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0
