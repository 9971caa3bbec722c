"""Pins for the oracle's reduced gradient, Gauss-Newton Hessian, PCG and
Newton solve (CPU only).  The references are finite differences of the
objective (Eq. (e:objective)), the dense Hessian assembled column by column
and solved by LAPACK, and the structure the paper states (Gauss-Newton
Hessian positive definite, compact perturbation of the identity after
preconditioning, divergence-free iterates for w = 0)."""
import numpy as np
import pytest

from oracle import spectral as S
from oracle import transport as T
from oracle.registration import Registration
from paper_1503_00757_gb300 import synth


def _problem(n=32, nt=8, **kw):
    mT, mR, vs = synth.blobs_pair(n, 1000)
    return Registration(mT, mR, nt, **kw), vs


def _fd(P, v, d, eps=1e-4):
    return (P.objective(v + eps * d)[0] - P.objective(v - eps * d)[0]) / (2 * eps)


@pytest.mark.parametrize("regnorm", [S.H1, S.H2])
def test_gradient_matches_fd_second_order_gamma0(regnorm):
    """gamma = 0: g is the L2 gradient of J; optimize-then-discretize gives an
    O(h_t^2) mismatch (observed order 2)."""
    rng = np.random.default_rng(0)
    errs = []
    for nt in (4, 8, 16):
        P, vs = _problem(nt=nt, regnorm=regnorm, beta_v=1e-3, beta_w=0.0)
        v = 0.5 * vs
        d = synth.velocity(32, 32, 6, 0.2, np.random.default_rng(1), grad_fraction=1.0)
        g, _ = P.gradient(v)
        fd = _fd(P, v, d)
        errs.append(abs(S.inner(g, d) - fd) / abs(fd))
    assert errs[-1] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_gradient_incompressible_along_divfree_directions():
    P, vs = _problem(nt=16, beta_v=1e-3, beta_w=np.inf)
    v = 0.5 * vs
    d = synth.velocity(32, 32, 6, 0.2, np.random.default_rng(2))
    g, _ = P.gradient(v)
    assert np.abs(S.div(g)).max() < 1e-10
    fd = _fd(P, v, d)
    assert abs(S.inner(g, d) - fd) / abs(fd) < 1e-3


@pytest.mark.parametrize("regnorm", [S.H1, S.H2])
def test_mass_source_gradient_is_projected_true_gradient(regnorm):
    """For 0 < beta_w < inf the reduced gradient equals K applied to the true
    gradient G of J with w = div v, so <g, d'> = <G, K d'> = FD of J along K d'.
    This pins K's mass-source form through the objective's w-term."""
    rng = np.random.default_rng(3)
    P, vs = _problem(nt=16, regnorm=regnorm, beta_v=1e-3, beta_w=1e-3)
    v = 0.5 * vs + synth.velocity(32, 32, 4, 0.2, rng, grad_fraction=1.0)
    dp = synth.velocity(32, 32, 6, 0.2, rng, grad_fraction=1.0)
    g, _ = P.gradient(v)
    d = S.apply_K(dp, regnorm, 1e-3, 1e-3)
    fd = _fd(P, v, d)
    assert abs(S.inner(g, dp) - fd) / abs(fd) < 2e-3


def test_gradient_without_image_force_is_regularization():
    P = Registration(np.full((16, 16), 0.3), np.full((16, 16), 0.3), 4, beta_v=0.05, beta_w=0.0)
    v = synth.velocity(16, 16, 3, 0.4, np.random.default_rng(4), grad_fraction=1.0)
    g, _ = P.gradient(v)
    assert np.abs(g - 0.05 * S.apply_A(v, S.H1)).max() < 1e-13


def _inverse_crime(n=32, nt=8, **kw):
    mT, _, vs = synth.blobs_pair(n, 1002)
    mR = T.state_solve(mT, vs, nt)[-1]
    return Registration(mT, mR, nt, **kw), vs


@pytest.mark.parametrize("beta_w", [0.0, np.inf])
def test_gn_hessian_matches_fd_of_gradient_at_zero_residual(beta_w):
    """At a zero-residual point lambda = 0, so Gauss-Newton equals the full
    Hessian and FD of g along v~ must match H v~ up to O(h_t^2)."""
    errs = []
    for nt in (4, 8, 16):
        P, vs = _inverse_crime(nt=nt, beta_v=1e-3, beta_w=beta_w)
        vt = synth.velocity(32, 32, 5, 0.2, np.random.default_rng(5), grad_fraction=0.0 if np.isinf(beta_w) else 1.0)
        eps = 1e-5
        gp, _ = P.gradient(vs + eps * vt)
        gm, _ = P.gradient(vs - eps * vt)
        P.gradient(vs)
        Hv = P.matvec(vt)
        errs.append(np.sqrt(S.inner(Hv - (gp - gm) / (2 * eps), Hv - (gp - gm) / (2 * eps)) / S.inner(Hv, Hv)))
    assert errs[-1] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_gn_hessian_symmetry_order_and_positivity():
    rng = np.random.default_rng(6)
    u = synth.velocity(32, 32, 6, 0.3, rng, grad_fraction=1.0)
    w = synth.velocity(32, 32, 6, 0.3, rng, grad_fraction=1.0)
    asym = []
    for nt in (4, 8, 16):
        P, vs = _problem(nt=nt, beta_v=1e-3, beta_w=0.0)
        P.gradient(0.5 * vs)
        Hu, Hw = P.matvec(u), P.matvec(w)
        a, b = S.inner(Hu, w), S.inner(u, Hw)
        asym.append(abs(a - b) / abs(a))
        assert S.inner(Hu, u) > 0 and S.inner(Hw, w) > 0
    assert asym[-1] < 1e-3
    assert asym[0] / asym[1] > 3.0 and asym[1] / asym[2] > 3.0


def test_pcg_matches_dense_solve_tiny_grid():
    """Assemble H column by column on an 8x8 grid (128 unknowns), solve with
    LAPACK, compare with PCG run to a tight tolerance.  Also checks that the
    preconditioned operator (beta_v A)^-1 H has eigenvalues >= ~1 off the
    k = 0 mode (compact perturbation of the identity, Appendix E)."""
    n, nt = 8, 4
    mT, mR, _ = synth.blobs_pair(n, 1003, vmax=0.3, kmax=2)
    P = Registration(mT, mR, nt, beta_v=1e-2, beta_w=0.0)
    g, _ = P.gradient(np.zeros((2, n, n)))
    N = 2 * n * n
    H = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        H[:, c] = P.matvec(e.reshape(2, n, n)).ravel()
    x_dense = np.linalg.solve(H, -g.ravel())
    x_pcg, it, relres, hit = P.pcg(g, 1e-12, 400)
    assert not hit
    assert np.linalg.norm(x_pcg.ravel() - x_dense) / np.linalg.norm(x_dense) < 1e-8
    Pinv = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        Pinv[:, c] = P.precond(e.reshape(2, n, n)).ravel()
    ev = np.linalg.eigvals(Pinv @ H)
    assert ev.real.min() > -1e-8
    assert np.sort(ev.real)[2:].min() > 1.0 - 1e-6  # two k=0 (translation) modes excepted
    assert np.abs(ev.imag).max() < 1e-3 * np.abs(ev).max()


@pytest.mark.parametrize("beta_w,regnorm", [(np.inf, S.H1), (0.0, S.H2), (1e-3, S.H1)])
def test_newton_solve_converges_and_decreases_J(beta_w, regnorm):
    mT, mR, vs = synth.blobs_pair(32, 1004, vmax=0.4, kmax=3)
    P = Registration(mT, mR, 8, regnorm=regnorm, beta_v=1e-2, beta_w=beta_w)
    v, st = P.solve(tol=1e-2)
    assert st["status"] == 0
    assert st["gnorm_rel"] <= 1e-2
    assert st["J"] < st["J0"]
    assert st["rnorm_rel_sq"] < 0.5
    if np.isinf(beta_w):
        assert np.abs(S.div(v)).max() < 1e-11
    assert st["n_pde"] == 2 * (st["n_newton"] + 1) + 2 * st["n_mv"] + st["n_ls"]


def test_newton_recovers_velocity_on_inverse_crime():
    n, nt = 32, 8
    mT, _, vs = synth.blobs_pair(n, 1005, vmax=0.3, kmax=2)
    mR = T.state_solve(mT, vs, nt)[-1]
    P = Registration(mT, mR, nt, beta_v=1e-5, beta_w=np.inf)
    v, st = P.solve(tol=1e-3)
    assert st["rnorm_rel_sq"] < 1e-3
    # the image only constrains v where grad m_T is not small; compare there
    gm = np.sqrt((S.grad(mT) ** 2).sum(0))
    mask = gm > 0.5 * gm.max()
    err = np.sqrt(((v - vs) ** 2).sum(0))[mask].mean() / np.sqrt((vs ** 2).sum(0))[mask].mean()
    assert err < 0.5


def test_cfl_policy():
    P, vs = _problem(n=64, nt=4)
    assert P.nt_for(vs, "fixed") == 4
    vmax = np.sqrt(vs[0] ** 2 + vs[1] ** 2).max()
    assert P.nt_for(vs, "cfl") == max(4, int(np.ceil(vmax * 64 / (2 * np.pi * 0.25))))
