"""GPU (CUDA, via the C ABI) vs FP64 oracle parity, element by element.

Tolerances: operator applications (spectral operators, objective, reduced
gradient, Gauss-Newton matvec) <= 1e-5 relative L2 in FP32; the end-to-end
solve <= 1e-3 relative in v and in the mismatch."""
import math

import numpy as np
import pytest

from oracle import spectral as S
from oracle import transport as T
from oracle.registration import Registration
from paper_1503_00757_gb300 import synth

from .gpu_util import check, check_rel, make_ctx, rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
U32 = 2.0 ** -24


def op_cond(beta_v, regnorm, x, y, b=None):
    """Conditioning of the sum y = beta_v A x + K b (reduced gradient, Hessian matvec):
    (||beta_v A x|| + ||b||) / ||y||.  A relative error e in the FP32 body force b passes
    through the projection K (a contraction) as an absolute error of at most e ||b||, so
    relative to ||y|| it is multiplied by this factor; it exceeds 1 where K removes most of
    b (Leray projection of a nearly curl-free force, mass source)."""
    ny = np.linalg.norm(y)
    terms = np.linalg.norm(beta_v * S.apply_A(x, regnorm)) + (np.linalg.norm(b) if b is not None else 0.0)
    return terms / ny


def op_tol(beta_v, regnorm, n1, n2, x, y, b=None, eta_max=1.0):
    """Tolerance for y = beta_v A x + K b: 1e-5 times max(1, op_cond), plus the FP32
    rounding bound of the regularization term, u * beta_v * max A^ * eta_max * ||x|| / ||y||,
    which matters where the H2 / H3 symbol |k|^4 / |k|^6 amplifies the rounding of the FP32
    operand (rounding the inputs alone moves the FP64 result that much).  eta_max: the largest
    viscosity of the shear model's second variation B = -div(2 eta (...)), which multiplies
    the same rounding (1 for the quadratic seminorms)."""
    Amax = S.reg_symbol(n1, n2, regnorm).max()
    ny = np.linalg.norm(y)
    return (OP_TOL * max(1.0, op_cond(beta_v, regnorm, x, y, b)) +
            U32 * beta_v * Amax * eta_max * np.linalg.norm(x) / ny)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00757_gb300.binding import lib
    lib()


def _field(n1, n2, seed, kmax=None):
    rng = np.random.default_rng(seed)
    kmax = kmax or min(n1, n2) // 4
    return synth.smooth_field(n1, n2, kmax, rng, decay=0.5) + 0.01 * rng.standard_normal((n1, n2))


GRIDS = [(16, 16), (64, 128), (128, 32), (256, 256)]


@pytest.mark.parametrize("n1,n2", GRIDS + [(1024, 1024)])
def test_spectral_grad_div(n1, n2):
    import torch
    ctx = make_ctx(n1, n2, 2)
    f = _field(n1, n2, 1)
    u = np.stack([_field(n1, n2, 2), _field(n1, n2, 3)])
    g = torch.empty(2, n1, n2, device="cuda")
    ctx.spectral_grad(to_gpu(f), g)
    d = torch.empty(n1, n2, device="cuda")
    ctx.spectral_div(to_gpu(u), d)
    check_rel("grad f", to_np(g), S.grad(f), OP_TOL)
    check_rel("div u", to_np(d), S.div(u), OP_TOL)


@pytest.mark.parametrize("n1,n2", GRIDS)
@pytest.mark.parametrize("regnorm,gamma", [(1, math.inf), (2, 0.0), (1, 1e-3), (2, 1e-3)])
def test_spectral_reg_proj_precond(n1, n2, regnorm, gamma):
    import torch
    beta = 1e-3
    ctx = make_ctx(n1, n2, 2, regnorm=regnorm, beta=beta, gamma=gamma)
    u = np.stack([_field(n1, n2, 4), _field(n1, n2, 5)])
    out = torch.empty(2, n1, n2, device="cuda")
    ctx.apply_reg(to_gpu(u), out)
    check_rel("beta_v A u", to_np(out), beta * S.apply_A(u, regnorm), OP_TOL)
    ctx.apply_proj(to_gpu(u), out)
    check_rel("K u", to_np(out), S.apply_K(u, regnorm, beta, gamma), OP_TOL)
    ctx.apply_precond(to_gpu(u), out)
    check_rel("(beta_v A)^-1 u", to_np(out), S.apply_precond(u, regnorm, beta), OP_TOL)


CASES = [
    # n1, n2, nt, regnorm, beta_v, beta_w, pair
    (64, 64, 4, 1, 1e-2, math.inf, "blobs"),
    (64, 64, 4, 2, 1e-2, 0.0, "blobs"),
    (64, 128, 8, 1, 1e-3, 1e-3, "blobs"),
    (128, 64, 8, 2, 1e-3, 1e-3, "labels"),
    (128, 128, 16, 1, 1e-3, math.inf, "ellipses"),
]


def _pair(kind, n1, n2, seed):
    if kind == "blobs":
        mT, mR, vs = synth.blobs_pair(max(n1, n2), seed)
    elif kind == "labels":
        mT, mR, vs = synth.labels_pair(max(n1, n2), seed, vmax=0.3)
    else:
        mT, mR, vs = synth.ellipses_pair(max(n1, n2), seed, vmax=0.2)
    # non-square grids subsample the square periodic images (they stay periodic and smooth)
    return _resample(mT, n1, n2), _resample(mR, n1, n2), _resample_v(vs, n1, n2)


def _resample(f, n1, n2):
    n = f.shape[0]
    return f[:: n // n1, :: n // n2] if (n1, n2) != f.shape else f


def _resample_v(v, n1, n2):
    return np.stack([_resample(v[0], n1, n2), _resample(v[1], n1, n2)])


def cfl_scaled(vs, n1, n2, nt, cfl=0.3):
    """Scale v so that max|v| nt^-1 / h_x = cfl.  Above ~0.3, Heun's per-step
    amplification of the highest modes, sqrt(1 + z^4/4) with z = pi * CFL,
    multiplies FP32 round-off by up to |.|^nt in every transport solve (the
    paper adapts nt to the CFL condition, Sec. 5.1)."""
    vmax = np.sqrt(vs[0] ** 2 + vs[1] ** 2).max()
    return vs * (cfl * 2 * np.pi * nt / (max(n1, n2) * vmax))


@pytest.mark.parametrize("case", CASES)
def test_objective_gradient_matvec(case):
    import torch
    n1, n2, nt, regnorm, bv, bw, kind = case
    mT, mR, vs = _pair(kind, n1, n2, 2000)
    v = cfl_scaled(vs, n1, n2, nt)
    vt = synth.velocity(n1, n2, min(n1, n2) // 8, 0.3, np.random.default_rng(7), grad_fraction=0.5)
    P = Registration(mT, mR, nt, regnorm=regnorm, beta_v=bv, beta_w=bw)
    ctx = make_ctx(n1, n2, nt, regnorm=regnorm, beta=bv, gamma=bw)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    m1 = torch.empty(n1, n2, device="cuda")
    J = ctx.objective(to_gpu(v), m1)
    J_ref, m_ref = P.objective(v)
    check_rel("m1", to_np(m1), m_ref[-1], OP_TOL)
    check("J", abs(J - J_ref) / abs(J_ref), OP_TOL)
    g = torch.empty(2, n1, n2, device="cuda")
    Jg = ctx.gradient(to_gpu(v), g)
    g_ref, _ = P.gradient(v)
    b = torch.empty(2, n1, n2, device="cuda")
    ctx.body_force(b)
    check_rel("b", to_np(b), P.b, OP_TOL)
    check("J (gradient call)", abs(Jg - J_ref) / abs(J_ref), OP_TOL)
    check_rel("g", to_np(g), g_ref, op_tol(bv, regnorm, n1, n2, v, g_ref, P.b), cond=op_cond(bv, regnorm, v, g_ref, P.b))
    Hv = torch.empty(2, n1, n2, device="cuda")
    ctx.hessian_matvec(to_gpu(vt), Hv)
    Hv_ref = P.matvec(vt)
    ctx.body_force(b)
    check_rel("b~", to_np(b), P.bt, OP_TOL)
    check_rel("H v~", to_np(Hv), Hv_ref, op_tol(bv, regnorm, n1, n2, vt, Hv_ref, P.bt),
              cond=op_cond(bv, regnorm, vt, Hv_ref, P.bt))
    ctx.close()


def test_degenerate_cases():
    import torch
    n = 16
    # constant images: no image force, g = beta_v A v exactly; zero velocity keeps m_T
    c = np.full((n, n), 0.25)
    ctx = make_ctx(n, n, 1, regnorm=1, beta=0.05, gamma=0.0)
    ctx.set_images(to_gpu(c), to_gpu(c))
    v = synth.velocity(n, n, 3, 0.4, np.random.default_rng(1), grad_fraction=1.0)
    g = torch.empty(2, n, n, device="cuda")
    J = ctx.gradient(to_gpu(v), g)
    assert rel_l2(to_np(g), 0.05 * S.apply_A(v, 1)) < OP_TOL
    m1 = torch.empty(n, n, device="cuda")
    ctx.objective(torch.zeros(2, n, n, device="cuda"), m1)
    assert np.abs(to_np(m1) - 0.25).max() < 1e-7
    assert J > 0
    ctx.close()


def test_matvec_before_gradient_is_state_error():
    import torch
    from paper_1503_00757_gb300.binding import RegError
    ctx = make_ctx(16, 16, 2)
    with pytest.raises(RegError) as e:
        ctx.hessian_matvec(torch.zeros(2, 16, 16, device="cuda"), torch.zeros(2, 16, 16, device="cuda"))
    assert e.value.status == 9
    ctx.close()


@pytest.mark.parametrize("n,nt", [(32, 4), (64, 8)])
def test_detgrad(n, nt):
    import torch
    vv = synth.velocity(n, n, 4, 0.5, np.random.default_rng(3), grad_fraction=0.5)
    ctx = make_ctx(n, n, nt)
    det = torch.empty(n, n, device="cuda")
    st = ctx.detgrad(to_gpu(vv), det)
    F1 = T.defgrad_solve(vv, nt)
    det_ref, D_ref = T.defgrad_measures(F1)
    check_rel("det F1", to_np(det), det_ref, OP_TOL)
    ref = (det_ref.min(), det_ref.mean(), det_ref.max(), D_ref.max(), D_ref.mean())
    for name, a, b in zip(("min det", "mean det", "max det", "max D", "mean D"), st, ref):
        check(name, abs(a - b) / max(1.0, abs(b)), 1e-5)
    # shear flow: det F1 = 1 exactly (Heun exact), D = |cos x2|
    X1, X2 = S.grid_coords(n, n)
    vsh = np.stack([np.sin(X2), np.zeros((n, n))])
    st = ctx.detgrad(to_gpu(vsh), det)
    assert np.abs(to_np(det) - 1).max() < 1e-5
    assert abs(st[3] - 1.0) < 1e-5
    ctx.close()


@pytest.mark.parametrize("s", [-0.5, 0.5])
def test_shear_gradient_matvec(s):
    import torch
    n1 = n2 = 64
    nt = 8
    mT, mR, vs = synth.blobs_pair(n1, 2001, vmax=0.4, kmax=3)
    v = 0.5 * vs
    vt = synth.velocity(n1, n2, 6, 0.3, np.random.default_rng(8))
    P = Registration(mT, mR, nt, regnorm=1, beta_v=1e-3, beta_w=math.inf, shear=s)
    ctx = make_ctx(n1, n2, nt, regnorm=1, beta=1e-3, gamma=math.inf, shear=s)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    g = torch.empty(2, n1, n2, device="cuda")
    J = ctx.gradient(to_gpu(v), g)
    g_ref, J_ref = P.gradient(v)
    check("J", abs(J - J_ref) / abs(J_ref), OP_TOL)
    check_rel("g", to_np(g), g_ref, op_tol(1e-3, 1, n1, n2, v, g_ref, P.b), cond=op_cond(1e-3, 1, v, g_ref, P.b))
    Hv = torch.empty(2, n1, n2, device="cuda")
    ctx.hessian_matvec(to_gpu(vt), Hv)
    Hv_ref = P.matvec(vt)
    b = torch.empty(2, n1, n2, device="cuda")
    ctx.body_force(b)
    check_rel("b~", to_np(b), P.bt, OP_TOL)
    check_rel("H v~", to_np(Hv), Hv_ref, op_tol(1e-3, 1, n1, n2, vt, Hv_ref, P.bt),
              cond=op_cond(1e-3, 1, vt, Hv_ref, P.bt))
    ctx.close()


@pytest.mark.parametrize("regnorm,gamma,shear", [(1, math.inf, 0.0), (2, 0.0, 0.0), (1, 1e-3, 0.0),
                                                 (1, math.inf, 0.5)])
def test_solve_end_to_end(regnorm, gamma, shear):
    import torch
    n, nt = 64, 4
    mT, mR, vs = synth.blobs_pair(n, 1000)
    P = Registration(mT, mR, nt, regnorm=regnorm, beta_v=1e-2, beta_w=gamma, shear=shear)
    v_ref, st_ref = P.solve(tol=1e-2)
    ctx = make_ctx(n, n, nt, regnorm=regnorm, beta=1e-2, gamma=gamma, shear=shear)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    v = torch.zeros(2, n, n, device="cuda")
    st = ctx.solve(v)
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2
    assert st["n_newton"] == st_ref["n_newton"]
    check_rel("solve v", to_np(v), v_ref, 1e-3)
    check("solve mismatch", abs(st["rnorm_rel_sq"] - st_ref["rnorm_rel_sq"]) / st_ref["rnorm_rel_sq"], 1e-3)
    ctx.close()


def test_graph_path_matches_direct_launches():
    """On a non-default stream every fixed launch sequence is captured once in a
    CUDA graph and replayed; results must equal the direct launches bit for bit."""
    import torch
    n, nt = 64, 8
    mT, mR, vs = synth.ellipses_pair(n, 2002, vmax=0.2)
    v = cfl_scaled(vs, n, n, nt)
    vt = synth.velocity(n, n, 6, 0.3, np.random.default_rng(9))
    outs = []
    for use_stream in (False, True):
        stream = torch.cuda.Stream() if use_stream else None
        ctx = make_ctx(n, n, nt, regnorm=1, beta=1e-3, gamma=math.inf)
        if stream is not None:
            ctx.set_stream(stream)
        with torch.cuda.stream(stream) if stream is not None else torch.cuda.stream(torch.cuda.current_stream()):
            ctx.set_images(to_gpu(mT), to_gpu(mR))
            g = torch.empty(2, n, n, device="cuda")
            Hv = torch.empty(2, n, n, device="cuda")
            vg = to_gpu(v)
            vtg = to_gpu(vt)
            for _ in range(2):  # second pass replays the captured graphs
                J = ctx.gradient(vg, g)
                ctx.hessian_matvec(vtg, Hv)
            vsol = torch.zeros(2, n, n, device="cuda")
            st = ctx.solve(vsol)
            torch.cuda.synchronize()
        outs.append((J, to_np(g), to_np(Hv), to_np(vsol), st["n_mv"]))
        ctx.close()
    (J0, g0, H0, v0, m0), (J1, g1, H1, v1, m1) = outs
    assert J0 == J1 and m0 == m1
    assert np.array_equal(g0, g1) and np.array_equal(H0, H1) and np.array_equal(v0, v1)


def test_warm_start_solve_matches_oracle():
    """Warm start (opts.warm_start): stopping test relative to g(0), forcing term
    relative to the gradient at the initial guess (Algorithm 2's g_0)."""
    import torch
    from paper_1503_00757_gb300.binding import default_opts
    n, nt = 64, 4
    mT, mR, vs = synth.blobs_pair(n, 1000)
    P = Registration(mT, mR, nt, regnorm=1, beta_v=1e-2, beta_w=math.inf)
    v0 = S.apply_K(0.3 * vs, 1, 1.0, math.inf)
    v_ref, st_ref = P.solve(v0=v0, tol=1e-2)
    ctx = make_ctx(n, n, nt, regnorm=1, beta=1e-2, gamma=math.inf)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    v = to_gpu(v0)
    st = ctx.solve(v, default_opts(tol=1e-2, warm_start=1))
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2
    assert st["n_newton"] == st_ref["n_newton"] and st["n_mv"] == st_ref["n_mv"]
    check_rel("warm-start solve v", to_np(v), v_ref, 1e-3)
    ctx.close()


@pytest.mark.parametrize("seed,gamma", [(4000, math.inf), (4013, math.inf), (4010, 0.0)])
def test_h2_solve_in_preconditioned_coordinates_matches_oracle(seed, gamma):
    """H2 solves iterate on y = (beta_v A')^(1/2) v (reg_solve): 128^2 mixed-batch pairs
    (nt=16, beta_v=1e-2) that stalled at the FP32 floor of the H2 gradient when iterating
    on v reach the tolerance with the FP64 oracle's Newton count and velocity."""
    import torch
    n, nt = 128, 16
    mT, mR, _ = synth.ellipses_pair(n, seed, vmax=0.196, kmax=16)
    P = Registration(mT, mR, nt, regnorm=2, beta_v=1e-2, beta_w=gamma)
    v_ref, st_ref = P.solve(tol=1e-2)
    assert st_ref["status"] == 0
    ctx = make_ctx(n, n, nt, regnorm=2, beta=1e-2, gamma=gamma)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    v = torch.zeros(2, n, n, device="cuda")
    st = ctx.solve(v)
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2
    assert st["n_newton"] == st_ref["n_newton"]
    check_rel("H2 solve v", to_np(v), v_ref, 1e-3)
    check("H2 solve mismatch", abs(st["rnorm_rel_sq"] - st_ref["rnorm_rel_sq"]) / st_ref["rnorm_rel_sq"], 1e-3)
    ctx.close()


@pytest.mark.parametrize("n,beta,gamma", [(256, 1e-3, 1e-3), (512, 1e-2, math.inf), (512, 1e-3, 0.0)])
def test_h2_solves_converge_at_full_size(n, beta, gamma):
    """Property at the 256^2 / 512^2 sizes (no oracle run): H2 solves of the mixed batch's
    settings reach ||g|| <= 1e-2 ||g(0)|| with a monotone objective and div v = 0 (w = 0)."""
    import torch
    from oracle import spectral as S
    nt = 16
    mT, mR, _ = synth.ellipses_pair(n, 4100 + n, vmax=0.049 * 512 / n, kmax=16)
    ctx = make_ctx(n, n, nt, regnorm=2, beta=beta, gamma=gamma)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    v = torch.zeros(2, n, n, device="cuda")
    st = ctx.solve(v)
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2
    assert st["J"] < st["J0"]
    if math.isinf(gamma):
        vn = to_np(v).astype(np.float64)
        assert np.abs(S.div(vn)).max() < 1e-4 * max(np.abs(vn).max(), 1e-30) * n
    ctx.close()


@pytest.mark.parametrize("n1,n2,regnorm,beta", [(64, 128, 2, 1e-2), (128, 64, 1, 1e-3), (32, 32, 2, 1e-3)])
def test_precond_sqrt(n1, n2, regnorm, beta):
    """Q^{+-1} x with Q^ = (beta_v A'^)^(1/2), A'(0) = 1, against the oracle's symbols; Q Q^-1 = I;
    Q^2 = the preconditioner's inverse (Q^-1 Q^-1 x = P^-1 x)."""
    import torch
    rng = np.random.default_rng(n1 + n2 + regnorm)
    x = np.stack([synth.gaussian_smooth(rng.standard_normal((n1, n2)), 0.05) for _ in range(2)])
    A = S.reg_symbol(n1, n2, regnorm).copy()
    A[0, 0] = 1.0
    Qs = np.sqrt(beta * A)
    ref = lambda m: np.stack([np.real(np.fft.ifft2(m * np.fft.fft2(x[c]))) for c in range(2)])
    ctx = make_ctx(n1, n2, 4, regnorm=regnorm, beta=beta)
    xg = to_gpu(x)
    out = torch.empty_like(xg)
    for inv, mult in ((False, Qs), (True, 1.0 / Qs)):
        ctx.apply_precond_sqrt(xg, out, inverse=inv)
        assert rel_l2(to_np(out), ref(mult)) < 1e-5
    back = torch.empty_like(xg)
    ctx.apply_precond_sqrt(xg, out, inverse=True)
    ctx.apply_precond_sqrt(out, back, inverse=False)
    # Q re-amplifies the FP32 rounding of Q^-1 x by up to max Q / min Q
    assert rel_l2(to_np(back), x) < 1e-5 + 2.0 ** -24 * Qs.max() / Qs.min()
    z = torch.empty_like(xg)
    ctx.apply_precond(xg, z)
    ctx.apply_precond_sqrt(xg, out, inverse=True)
    ctx.apply_precond_sqrt(out, back, inverse=True)
    assert rel_l2(to_np(back), to_np(z)) < 1e-5
    ctx.close()


def test_precision_config_full_size():
    """The precision workload at its full size: 256^2 smoothed noisy 4-label images, v* with
    |k| <= 8 and a 30 % gradient part (max|v*| = 0.8), H2, beta_v = beta_w = 1e-3 (mass source).
    Operator parity against the FP64 oracle at v = v*/2 with nt adapted to CFL 0.25 (66 steps);
    then the GPU solve with the CFL policy reaches the tolerance within 100 Newton iterations
    (property, no oracle solve)."""
    import torch
    from paper_1503_00757_gb300.binding import default_opts
    n = 256
    mT, mR, vs = synth.labels_pair(n, 2000)
    v = 0.5 * vs
    vmax = np.sqrt(v[0] ** 2 + v[1] ** 2).max()
    nt = int(math.ceil(vmax * n / (2 * math.pi * 0.25)))
    assert 60 <= nt <= 70
    vt = synth.velocity(n, n, 8, 0.3, np.random.default_rng(9), grad_fraction=0.3)
    P = Registration(mT, mR, nt, regnorm=2, beta_v=1e-3, beta_w=1e-3)
    ctx = make_ctx(n, n, nt, regnorm=2, beta=1e-3, gamma=1e-3)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    g = torch.empty(2, n, n, device="cuda")
    J = ctx.gradient(to_gpu(v), g)
    g_ref, J_ref = P.gradient(v)
    check("J", abs(J - J_ref) / abs(J_ref), OP_TOL)
    b = torch.empty(2, n, n, device="cuda")
    ctx.body_force(b)
    check_rel("b", to_np(b), P.b, OP_TOL)
    check_rel("g", to_np(g), g_ref, op_tol(1e-3, 2, n, n, v, g_ref, P.b), cond=op_cond(1e-3, 2, v, g_ref, P.b))
    Hv = torch.empty(2, n, n, device="cuda")
    ctx.hessian_matvec(to_gpu(vt), Hv)
    Hv_ref = P.matvec(vt)
    ctx.body_force(b)
    # the intermediate b~ carries the FP32 rounding of 2 nt RK2 stages (incremental state and
    # adjoint): its bound grows with nt beyond the 32 steps of the other cases
    check_rel("b~", to_np(b), P.bt, OP_TOL * max(1.0, nt / 32))
    check_rel("H v~", to_np(Hv), Hv_ref, op_tol(1e-3, 2, n, n, vt, Hv_ref, P.bt), cond=op_cond(1e-3, 2, vt, Hv_ref, P.bt))
    ctx.close()
    ctx = make_ctx(n, n, 16, regnorm=2, beta=1e-3, gamma=1e-3)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    vsol = torch.zeros(2, n, n, device="cuda")
    # a hard problem (H2, beta_v = 1e-3, displacements up to 0.8): on one GB300 it takes 67
    # Newton iterations and ~6200 matvecs, most PCG solves at their 100-iteration cap
    st = ctx.solve(vsol, default_opts(tol=1e-2, nt_policy=1, cfl_max=0.25, maxit_newton=100))
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2 and st["J"] < st["J0"]
    assert st["cfl"] <= 0.25 + 1e-9 and st["nt_used"] >= 16
    ctx.close()


def test_registration_workload_at_full_size():
    """The benchmark's registration workload at its full size, in the launch configuration the
    benchmark times. Workload: 512^2, nt = 32, H1, incompressible, beta_v = 1e-3, its first
    seeded image pair. Launch configuration: 4 rows per row CTA, 2 columns per column CTA,
    operand prefetch, programmatic dependent launch, CUDA graphs on a non-default stream.

    Element by element against the FP64 oracle: the state solve (m_1 and J).

    Properties that hold at any size:
    * the reduced gradient against central differences of J, in the L2 inner product of the
      grid (weight h1 h2);
    * the Gauss-Newton matvec against central differences of the gradient at a zero-residual
      point (m_R := m_1(v)), where Gauss-Newton equals the full Hessian;
    * linearity of the matvec: exact for a factor 2, to FP32 rounding for a sum.

    Tolerances. The oracle's own mismatch of the two difference checks at this size is
    1.5e-4 (gradient) and 8.5e-5 (matvec): the O(h_t^2) consistency of the
    optimize-then-discretize derivatives. FP32 rounding adds about 1e-5 to the differences."""
    import torch
    from paper_1503_00757_gb300.binding import Context
    n, nt, beta = 512, 32, 1e-3
    mT, mR, vs = synth.ellipses_pair(n, 3000, vmax=0.098)
    v = 0.5 * vs
    vt = synth.velocity(n, n, 16, 0.3, np.random.default_rng(7))
    w = synth.velocity(n, n, 8, 0.2, np.random.default_rng(8), grad_fraction=0.5)
    J_ref, m_ref = Registration(mT, mR, nt, regnorm=1, beta_v=beta, beta_w=math.inf).objective(v)

    stream = torch.cuda.Stream()
    ctx = Context(n, n, nt, regnorm=1, beta=beta, gamma=math.inf, stream=stream)
    ctx.set_tiles(4, 2, 1)
    ctx.set_pdl(True)
    mTd, mRd, vd, vtd, wd = to_gpu(mT), to_gpu(mR), to_gpu(v), to_gpu(vt), to_gpu(w)
    m1 = torch.empty(n, n, device="cuda")
    g = torch.empty(2, n, n, device="cuda")
    torch.cuda.synchronize()
    ctx.set_images(mTd, mRd)
    J = ctx.objective(vd, m1)
    stream.synchronize()
    assert rel_l2(to_np(m1), m_ref[-1]) < OP_TOL
    assert abs(J - J_ref) < OP_TOL * abs(J_ref)

    # gradient vs central differences of J along d = g / |g|. Every device input is made on
    # the default stream and synchronized before the context's stream reads it.
    h2 = (2 * math.pi / n) ** 2
    ctx.gradient(vd, g)
    stream.synchronize()
    gn = to_np(g)
    d = gn / np.linalg.norm(gn)
    eps = 1e-2 * np.linalg.norm(v)
    vp, vm = to_gpu(v + eps * d), to_gpu(v - eps * d)
    torch.cuda.synchronize()
    Jp = ctx.objective(vp)
    Jm = ctx.objective(vm)
    fd = (Jp - Jm) / (2 * eps)
    gd = h2 * float(np.sum(gn * d))
    assert abs(fd - gd) < 2e-3 * abs(gd), (fd, gd)

    # zero residual: m_R := m_1(v); matvecs at v, then central differences of the gradient
    e = 1e-2 * np.linalg.norm(v) / np.linalg.norm(vt)
    mR0 = m1.clone()
    vt2, vtw = 2.0 * vtd, vtd + wd
    vep, vem = to_gpu(v + e * vt), to_gpu(v - e * vt)
    Hv, H2v, Hw, Hvw = (torch.empty(2, n, n, device="cuda") for _ in range(4))
    gp, gm = torch.empty_like(g), torch.empty_like(g)
    torch.cuda.synchronize()
    ctx.set_images(mTd, mR0)
    ctx.gradient(vd, g)
    ctx.hessian_matvec(vtd, Hv)
    ctx.hessian_matvec(vt2, H2v)
    ctx.hessian_matvec(wd, Hw)
    ctx.hessian_matvec(vtw, Hvw)
    stream.synchronize()
    assert torch.equal(H2v, 2.0 * Hv)
    assert rel_l2(to_np(Hvw), to_np(Hv) + to_np(Hw)) < OP_TOL
    ctx.gradient(vep, gp)
    ctx.gradient(vem, gm)
    stream.synchronize()
    fdH = (to_np(gp) - to_np(gm)) / (2 * e)
    assert rel_l2(fdH, to_np(Hv)) < 1e-3
    ctx.close()


def test_register_host_matches_oracle():
    """reg_register_host (host buffers: the images are copied in, the velocity copied out)
    solves the plain 64^2 problem like the FP64 oracle: same Newton count, v and mismatch
    to 1e-3.  A second call on the same context with a warm start from the first solution
    (host buffer) converges at once (the stopping test stays relative to g(0))."""
    import torch
    from paper_1503_00757_gb300.binding import default_opts
    n, nt = 64, 4
    mT, mR, vs = synth.blobs_pair(n, 1000)
    P = Registration(mT, mR, nt, regnorm=1, beta_v=1e-2, beta_w=math.inf)
    v_ref, st_ref = P.solve(tol=1e-2)
    stream = torch.cuda.Stream()
    ctx = make_ctx(n, n, nt, regnorm=1, beta=1e-2, gamma=math.inf)
    ctx.set_stream(stream)
    hT = torch.from_numpy(mT.astype(np.float32)).pin_memory()
    hR = torch.from_numpy(mR.astype(np.float32)).pin_memory()
    hv = torch.full((2, n, n), float("nan"), dtype=torch.float32).pin_memory()
    st = ctx.register_host(hT, hR, hv)
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2
    assert st["n_newton"] == st_ref["n_newton"]
    check_rel("register_host v", hv.numpy(), v_ref, 1e-3)
    check("register_host mismatch", abs(st["rnorm_rel_sq"] - st_ref["rnorm_rel_sq"]) / st_ref["rnorm_rel_sq"], 1e-3)
    # numpy host buffers (pageable), warm start from the solution just returned
    hv2 = hv.numpy().copy()
    st2 = ctx.register_host(mT.astype(np.float32), mR.astype(np.float32), hv2, default_opts(tol=1e-2, warm_start=1))
    assert st2["status"] == 0 and st2["n_newton"] == 0 and st2["gnorm_rel"] <= 1e-2
    assert np.array_equal(hv2, hv.numpy())
    ctx.close()
