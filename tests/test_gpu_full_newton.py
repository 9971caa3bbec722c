"""Full-Newton Hessian and the H3 seminorm on the GPU against the FP64 oracle.

Full Newton (reg_set_hessian): the incremental adjoint keeps its source -div(lam v~) and the
incremental body force its term lam grad m~ (Eq. (e:inc-adj-eq-elim) and the second variations
of Sec. 3.2, which the Gauss-Newton approximation drops).  Compared element by element with the
oracle's full matvec at a nonzero residual (where it differs from Gauss-Newton by O(lam)): b~
and H v~, for H1 incompressible, H2 with a mass source and the shear model; then a full-Newton
solve against the oracle's.  H3 (symbol |k|^6): the spectral operators, and a solve (which runs
in preconditioned coordinates) against the oracle's solve.  Tolerances as in test_gpu_parity."""
import math

import numpy as np
import pytest

from oracle import spectral as S
from oracle.registration import Registration
from paper_1503_00757_gb300 import synth

from .gpu_util import check, check_rel, make_ctx, to_gpu, to_np
from .test_gpu_parity import OP_TOL, cfl_scaled, op_cond, op_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00757_gb300.binding import lib
    lib()


CASES = [
    # n, nt, regnorm, beta_v, beta_w, shear
    (64, 8, 1, 1e-2, math.inf, 0.0),
    (64, 8, 2, 1e-3, 1e-3, 0.0),
    (64, 8, 1, 1e-3, math.inf, 0.5),  # shear (nu = 3); at 128^2 FP32 input rounding alone moves H v~ by 1.2e-5
    (128, 8, 1, 1e-3, 0.0, 0.0),
]


@pytest.mark.parametrize("case", CASES)
def test_full_newton_matvec_matches_oracle(case):
    import torch
    n, nt, regnorm, bv, bw, sh = case
    mT, mR, vs = synth.blobs_pair(n, 2400 + n, vmax=0.4, kmax=3)
    v = 0.5 * cfl_scaled(vs, n, n, nt, cfl=0.25)
    vt = synth.velocity(n, n, max(2, n // 8), 0.3, np.random.default_rng(5), grad_fraction=0.0 if sh else 0.5)
    P = Registration(mT, mR, nt, regnorm=regnorm, beta_v=bv, beta_w=bw, shear=sh, hessian="full")
    g_ref, _ = P.gradient(v)
    Hv_ref = P.matvec(vt)
    Pg = Registration(mT, mR, nt, regnorm=regnorm, beta_v=bv, beta_w=bw, shear=sh)
    Pg.gradient(v)
    Hgn = Pg.matvec(vt)
    ctx = make_ctx(n, n, nt, regnorm=regnorm, beta=bv, gamma=bw, shear=sh)
    ctx.set_hessian(True)
    assert ctx.transport_config()[0] == 0
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    g = torch.empty(2, n, n, device="cuda")
    Hv = torch.empty(2, n, n, device="cuda")
    bt = torch.empty(2, n, n, device="cuda")
    ctx.gradient(to_gpu(v), g)
    ctx.hessian_matvec(to_gpu(vt), Hv)
    ctx.body_force(bt)
    torch.cuda.synchronize()
    # the case is one where the lambda terms matter
    assert np.linalg.norm(Hv_ref - Hgn) > 1e-2 * np.linalg.norm(Hv_ref)
    check_rel("b~ (full Newton)", to_np(bt), P.bt, OP_TOL)
    from oracle import shear as SH
    eta_max = float(SH.viscosity(v, SH.nu_from_shear(sh)).max()) if sh else 1.0
    check_rel("H v~ (full Newton)", to_np(Hv), Hv_ref, op_tol(bv, regnorm, n, n, vt, Hv_ref, P.bt, eta_max),
              cond=op_cond(bv, regnorm, vt, Hv_ref, P.bt), eta_max=eta_max)
    # back to Gauss-Newton on the same context
    ctx.set_hessian(False)
    ctx.gradient(to_gpu(v), g)
    ctx.hessian_matvec(to_gpu(vt), Hv)
    torch.cuda.synchronize()
    check_rel("H v~ (Gauss-Newton after full)", to_np(Hv), Hgn, op_tol(bv, regnorm, n, n, vt, Hgn, Pg.bt, eta_max),
              cond=op_cond(bv, regnorm, vt, Hgn, Pg.bt), eta_max=eta_max)
    ctx.close()


def test_full_newton_solve_matches_oracle():
    import torch
    n, nt = 64, 4
    mT, mR, _ = synth.blobs_pair(n, 1000)
    P = Registration(mT, mR, nt, regnorm=1, beta_v=1e-2, beta_w=math.inf, hessian="full")
    v_ref, st_ref = P.solve(tol=1e-3)
    assert st_ref["status"] == 0
    ctx = make_ctx(n, n, nt, regnorm=1, beta=1e-2, gamma=math.inf)
    ctx.set_hessian(True)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    v = torch.zeros(2, n, n, device="cuda")
    from paper_1503_00757_gb300.binding import default_opts
    st = ctx.solve(v, default_opts(tol=1e-3))
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-3
    assert st["n_newton"] == st_ref["n_newton"]
    check_rel("full-Newton solve v", to_np(v), v_ref, 1e-3)
    ctx.close()


@pytest.mark.parametrize("gamma", [math.inf, 0.0, 1e-2])
def test_h3_operators_match_oracle(gamma):
    import torch
    n, beta = 64, 1e-3
    rng = np.random.default_rng(17)
    u = np.stack([synth.smooth_field(n, n, 8, rng, decay=0.5) for _ in range(2)])
    ctx = make_ctx(n, n, 2, regnorm=3, beta=beta, gamma=gamma)
    out = torch.empty(2, n, n, device="cuda")
    ctx.apply_reg(to_gpu(u), out)
    ref = beta * S.apply_A(u, S.H3)
    check_rel("beta_v A u (H3)", to_np(out), ref, op_tol(beta, 3, n, n, u, ref))
    ctx.apply_proj(to_gpu(u), out)
    check_rel("K u (H3)", to_np(out), S.apply_K(u, S.H3, beta, gamma), OP_TOL)
    ctx.apply_precond(to_gpu(u), out)
    check_rel("(beta_v A)^-1 u (H3)", to_np(out), S.apply_precond(u, S.H3, beta), OP_TOL)
    ctx.close()


@pytest.mark.parametrize("gamma", [math.inf, 1e-3])
def test_h3_solve_matches_oracle(gamma):
    import torch
    n, nt = 64, 4
    mT, mR, _ = synth.blobs_pair(n, 1000)
    P = Registration(mT, mR, nt, regnorm=S.H3, beta_v=1e-4, beta_w=gamma)
    v_ref, st_ref = P.solve(tol=1e-2)
    assert st_ref["status"] == 0
    ctx = make_ctx(n, n, nt, regnorm=3, beta=1e-4, gamma=gamma)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    v = torch.zeros(2, n, n, device="cuda")
    st = ctx.solve(v)
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2
    assert st["n_newton"] == st_ref["n_newton"]
    check_rel("H3 solve v", to_np(v), v_ref, 1e-3)
    check("H3 solve mismatch", abs(st["rnorm_rel_sq"] - st_ref["rnorm_rel_sq"]) / st_ref["rnorm_rel_sq"], 1e-3)
    ctx.close()
