"""The cluster-resident transport kernel (one launch per transport solve, row spectra kept in
shared memory, column slabs exchanged through distributed shared memory) against the FP64
oracle element by element, and against the two-kernel path, on every square grid it serves
below the benchmark's 512^2 (which test_gpu_parity_full covers): 16^2 .. 128^2 on one CTA,
256^2 on a cluster of 4.  Quantities: m_1, J (state solve), b and g (adjoint solve, body
force, reduced gradient), b~ and H v~ (incremental state and adjoint, Gauss-Newton matvec).
Tolerances as in test_gpu_parity."""
import math

import numpy as np
import pytest

from oracle.registration import Registration
from paper_1503_00757_gb300 import synth

from .gpu_util import check, check_rel, to_gpu, to_np
from .test_gpu_parity import OP_TOL, cfl_scaled, op_cond, op_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00757_gb300.binding import lib
    lib()


def _run(ctx, n, mT, mR, v, vt):
    import torch
    m1 = torch.empty(n, n, device="cuda")
    g, b, Hv, bt = (torch.empty(2, n, n, device="cuda") for _ in range(4))
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    J = ctx.objective(to_gpu(v), m1)
    ctx.gradient(to_gpu(v), g)
    ctx.body_force(b)
    ctx.hessian_matvec(to_gpu(vt), Hv)
    ctx.body_force(bt)
    torch.cuda.synchronize()
    return dict(J=J, m1=to_np(m1), g=to_np(g), b=to_np(b), Hv=to_np(Hv), bt=to_np(bt))


CASES = [
    # n, nt, regnorm, beta_v, beta_w
    (16, 8, 1, 1e-2, math.inf),
    (32, 4, 2, 1e-2, 0.0),
    (64, 8, 1, 1e-3, 1e-3),
    (128, 16, 1, 1e-3, math.inf),
    (128, 8, 2, 1e-3, 1e-3),
    (256, 8, 1, 1e-3, math.inf),
    (256, 4, 2, 1e-2, 0.0),
]


@pytest.mark.parametrize("case", CASES)
def test_cluster_transport_matches_oracle_and_two_kernel_path(case):
    from paper_1503_00757_gb300.binding import Context
    n, nt, regnorm, bv, bw = case
    # smooth blob images below 128^2 (the ellipse images' edges are unresolved there), ellipses above
    if n <= 64:
        mT, mR, vs = synth.blobs_pair(n, 2200 + n, vmax=0.2, kmax=2)
    else:
        mT, mR, vs = synth.ellipses_pair(n, 2200 + n, vmax=0.2, kmax=max(2, n // 16))
    v = 0.5 * cfl_scaled(vs, n, n, nt, cfl=0.25)  # half the displacement: lam = m_R - m_1 does not cancel
    vt = synth.velocity(n, n, max(2, n // 8), 0.3, np.random.default_rng(n + 3), grad_fraction=0.5)
    P = Registration(mT, mR, nt, regnorm=regnorm, beta_v=bv, beta_w=bw)
    J_ref, m_ref = P.objective(v)
    g_ref, _ = P.gradient(v)
    b_ref = P.b.copy()
    Hv_ref = P.matvec(vt)
    bt_ref = P.bt.copy()

    ctx = Context(n, n, nt, regnorm=regnorm, beta=bv, gamma=bw)
    ctx.set_transport(True)
    use, cs, active = ctx.transport_config()
    assert use == 1 and cs == max(1, n * n // 16384) and active >= 1
    out = _run(ctx, n, mT, mR, v, vt)
    ctx.set_transport(False)
    assert ctx.transport_config()[0] == 0
    two = _run(ctx, n, mT, mR, v, vt)
    ctx.close()

    # the two transport paths agree to FP32 rounding
    for k in ("m1", "b", "bt"):
        check_rel(f"{k}: cluster vs two-kernel", out[k], two[k], OP_TOL)
    for tag, res in ((" (two-kernel path)", two), ("", out)):
        check_rel("m1" + tag, res["m1"], m_ref[-1], OP_TOL)
        check("J" + tag, abs(res["J"] - J_ref) / abs(J_ref), OP_TOL)
        check_rel("b" + tag, res["b"], b_ref, OP_TOL)
        check_rel("g" + tag, res["g"], g_ref, op_tol(bv, regnorm, n, n, v, g_ref, b_ref),
                  cond=op_cond(bv, regnorm, v, g_ref, b_ref))
        check_rel("b~" + tag, res["bt"], bt_ref, OP_TOL)
        check_rel("H v~" + tag, res["Hv"], Hv_ref, op_tol(bv, regnorm, n, n, vt, Hv_ref, bt_ref),
                  cond=op_cond(bv, regnorm, vt, Hv_ref, bt_ref))


def test_cluster_solve_matches_oracle_solve():
    """A full registration (Algorithm 1) on each transport path reaches the tolerance with the
    FP64 oracle's Newton count, and the FP64 oracle confirms the stopping test at the GPU's
    velocity: ||g(v)|| <= 1e-3 ||g(0)|| with g evaluated by the oracle (slack 10 % for the FP32
    gradient the GPU stopped on, whose error is ~1e-5 ||g(0)||).

    The velocity itself is fixed only to the stopping rule: two iterates that both satisfy
    ||g|| <= 1e-3 ||g(0)|| may differ by up to ||H^-1|| 2e-3 ||g(0)||, i.e. by kappa(H) 2e-3
    relative, and the paths' FP32 roundings send PCG down slightly different iterates (measured
    1.0e-3 for the two-kernel path and 1.6e-3 for the cluster path against the oracle's solve),
    so v is compared at 3e-3 as a sanity bound; the gradient check is the one that binds."""
    import torch
    from paper_1503_00757_gb300.binding import Context, default_opts
    n, nt = 128, 16
    mT, mR, _ = synth.ellipses_pair(n, 3100, vmax=0.2)
    P = Registration(mT, mR, nt, regnorm=1, beta_v=1e-3, beta_w=math.inf)
    v_ref, st_ref = P.solve(tol=1e-3)
    assert st_ref["status"] == 0
    g0 = np.linalg.norm(P.gradient(np.zeros_like(v_ref))[0])
    for cluster in (True, False):
        ctx = Context(n, n, nt, regnorm=1, beta=1e-3, gamma=math.inf)
        ctx.set_transport(cluster)
        ctx.set_images(to_gpu(mT), to_gpu(mR))
        v = torch.zeros(2, n, n, device="cuda")
        st = ctx.solve(v, default_opts(tol=1e-3))
        torch.cuda.synchronize()
        ctx.close()
        tag = "cluster" if cluster else "two-kernel"
        assert st["status"] == 0 and st["gnorm_rel"] <= 1e-3
        assert st["n_newton"] == st_ref["n_newton"]
        vg = to_np(v).astype(np.float64)
        g_rel = np.linalg.norm(P.gradient(vg)[0]) / g0
        check(f"oracle ||g(v)|| / ||g(0)|| at the solved v ({tag} path)", g_rel, 1.1e-3)
        check_rel(f"solve v ({tag} path), stopping-rule spread", vg, v_ref, 3e-3)
