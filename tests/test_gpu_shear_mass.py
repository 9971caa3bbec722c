"""The nonlinear Stokes (shear) model with a mass source (App. A.2) and without a constraint
(gamma = 0) on the GPU against the FP64 oracle: objective, reduced gradient, Gauss-Newton
matvec element by element, and a full solve (Newton count, v and mismatch to 1e-3).
Tolerances as in test_gpu_parity, the rounding term carrying the largest viscosity."""
import math

import numpy as np
import pytest

from oracle import shear as SH
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


@pytest.mark.parametrize("s,bw", [(0.5, 1e-2), (-0.5, 1e-2), (0.5, 0.0)])
def test_shear_mass_source_gradient_matvec(s, bw):
    import torch
    n, nt, bv = 64, 8, 1e-2
    mT, mR, vs = synth.blobs_pair(n, 2600, vmax=0.4, kmax=3)
    v = 0.5 * cfl_scaled(vs, n, n, nt, cfl=0.25) + synth.velocity(n, n, 3, 0.05, np.random.default_rng(3),
                                                                   grad_fraction=1.0)
    vt = synth.velocity(n, n, 6, 0.3, np.random.default_rng(4), grad_fraction=0.5)
    P = Registration(mT, mR, nt, regnorm=1, beta_v=bv, beta_w=bw, shear=s)
    J_ref, _ = P.objective(v)
    g_ref, _ = P.gradient(v)
    b_ref = P.b.copy()
    Hv_ref = P.matvec(vt)
    ctx = make_ctx(n, n, nt, regnorm=1, beta=bv, gamma=bw, shear=s)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    g = torch.empty(2, n, n, device="cuda")
    Hv = torch.empty(2, n, n, device="cuda")
    J = ctx.objective(to_gpu(v))
    ctx.gradient(to_gpu(v), g)
    ctx.hessian_matvec(to_gpu(vt), Hv)
    torch.cuda.synchronize()
    eta_max = float(SH.viscosity(v, SH.nu_from_shear(s)).max())
    check("J", abs(J - J_ref) / abs(J_ref), OP_TOL)
    check_rel("g", to_np(g), g_ref, op_tol(bv, 1, n, n, v, g_ref, b_ref, eta_max), cond=op_cond(bv, 1, v, g_ref, b_ref),
              eta_max=eta_max)
    check_rel("H v~", to_np(Hv), Hv_ref, op_tol(bv, 1, n, n, vt, Hv_ref, P.bt, eta_max),
              cond=op_cond(bv, 1, vt, Hv_ref, P.bt), eta_max=eta_max)
    ctx.close()


def test_shear_mass_source_solve_matches_oracle():
    import torch
    n, nt = 64, 8
    mT, mR, _ = synth.blobs_pair(n, 1000)
    P = Registration(mT, mR, nt, regnorm=1, beta_v=1e-2, beta_w=1e-2, shear=0.5)
    v_ref, st_ref = P.solve(tol=1e-2)
    assert st_ref["status"] == 0
    ctx = make_ctx(n, n, nt, regnorm=1, beta=1e-2, gamma=1e-2, shear=0.5)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    v = torch.zeros(2, n, n, device="cuda")
    st = ctx.solve(v)
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2
    assert st["n_newton"] == st_ref["n_newton"]
    check_rel("shear + mass source solve v", to_np(v), v_ref, 1e-3)
    check("shear + mass source mismatch", abs(st["rnorm_rel_sq"] - st_ref["rnorm_rel_sq"]) / st_ref["rnorm_rel_sq"], 1e-3)
    ctx.close()
