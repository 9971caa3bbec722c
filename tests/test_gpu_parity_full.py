"""Element-by-element parity with the FP64 oracle at the sizes the benchmark times.

* 512^2, nt = 32: the registration workload (its first seeded pair, H1, incompressible,
  beta_v = 1e-3) at a linearization point v = v*/2 and a band-limited direction v~.  The
  state, adjoint, body force, reduced gradient, incremental state and adjoint, incremental
  body force and Gauss-Newton matvec are compared with the oracle element by element, in
  the launch configurations the benchmark uses.
* 1024^2: the same quantities at a small nt (the oracle's cost grows with nt), which runs
  the 1024-point row kernels (no operand prefetch, two CTAs per SM) and the 1024-point
  column pass that the 1024^2 matvec measurement times.

Tolerances as in test_gpu_parity: 1e-5 relative L2 for m_1, J, b, b~; for g and H v~ 1e-5
times the conditioning factor of the sum beta_v A x + K b (op_cond)."""
import math

import numpy as np
import pytest

from oracle.registration import Registration
from paper_1503_00757_gb300 import synth

from .gpu_util import check, check_rel, to_gpu, to_np
from .test_gpu_parity import OP_TOL, op_cond, op_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00757_gb300.binding import lib
    lib()


def _oracle(n, nt, seed, vmax, beta):
    mT, mR, vs = synth.ellipses_pair(n, seed, vmax=vmax)
    v = 0.5 * vs
    vt = synth.velocity(n, n, 16, 0.3, np.random.default_rng(7))
    P = Registration(mT, mR, nt, regnorm=1, beta_v=beta, beta_w=math.inf)
    J_ref, m_ref = P.objective(v)
    g_ref, _ = P.gradient(v)
    b_ref = P.b.copy()
    Hv_ref = P.matvec(vt)
    return dict(n=n, nt=nt, beta=beta, mT=mT, mR=mR, v=v, vt=vt, J=J_ref, m1=m_ref[-1], g=g_ref, b=b_ref,
                Hv=Hv_ref, bt=P.bt.copy())


@pytest.fixture(scope="module")
def ref512():
    # the benchmark's workload: 512^2, nt = 32, first pair (seed 3000), max|v*| = 0.098 (CFL 0.25)
    return _oracle(512, 32, 3000, 0.098, 1e-3)


@pytest.fixture(scope="module")
def ref1024():
    # 1024^2 at nt = 4, max|v*| scaled for CFL 0.25 at that nt
    nt = 4
    return _oracle(1024, nt, 3000, 0.25 * 2 * math.pi * nt / 1024 * 2, 1e-3)


def _compare(R, configure):
    """Run the GPU path (a context on a non-default stream, configured by `configure`)
    on the oracle's inputs and check every intermediate element by element."""
    import torch
    from paper_1503_00757_gb300.binding import Context
    n, nt, beta = R["n"], R["nt"], R["beta"]
    stream = torch.cuda.Stream()
    ctx = Context(n, n, nt, regnorm=1, beta=beta, gamma=math.inf, stream=stream)
    configure(ctx)
    mTd, mRd, vd, vtd = to_gpu(R["mT"]), to_gpu(R["mR"]), to_gpu(R["v"]), to_gpu(R["vt"])
    m1 = torch.empty(n, n, device="cuda")
    g = torch.empty(2, n, n, device="cuda")
    b = torch.empty(2, n, n, device="cuda")
    Hv = torch.empty(2, n, n, device="cuda")
    bt = torch.empty(2, n, n, device="cuda")
    torch.cuda.synchronize()
    ctx.set_images(mTd, mRd)
    J = ctx.objective(vd, m1)
    Jg = ctx.gradient(vd, g)
    ctx.body_force(b)
    # twice: the second call replays the captured launch sequence
    for _ in range(2):
        ctx.hessian_matvec(vtd, Hv)
    ctx.body_force(bt)
    stream.synchronize()
    check_rel("m1", to_np(m1), R["m1"], OP_TOL)
    check("J", abs(J - R["J"]) / abs(R["J"]), OP_TOL)
    check("J (gradient call)", abs(Jg - R["J"]) / abs(R["J"]), OP_TOL)
    check_rel("b", to_np(b), R["b"], OP_TOL)
    check_rel("g", to_np(g), R["g"], op_tol(beta, 1, n, n, R["v"], R["g"], R["b"]),
              cond=op_cond(beta, 1, R["v"], R["g"], R["b"]))
    check_rel("b~", to_np(bt), R["bt"], OP_TOL)
    check_rel("H v~", to_np(Hv), R["Hv"], op_tol(beta, 1, n, n, R["vt"], R["Hv"], R["bt"]),
              cond=op_cond(beta, 1, R["vt"], R["Hv"], R["bt"]))
    ctx.close()


# launch configurations of the 512^2 registration workload: the cluster-resident transport
# kernel (the default on this grid), and the row/column kernel pairs with the tiles and launch
# mode the autotuner has chosen on a GB300 (4 rows per row CTA, 2 spectrum columns per column
# CTA, operand prefetch, with and without programmatic dependent launch)
CONFIGS_512 = {
    "cluster transport": dict(transport=True, pdl=True),
    "two-pass R4 C2 prefetch pdl": dict(transport=False, tiles=(4, 2, 1), pdl=True),
    "two-pass R4 C2 prefetch no-pdl": dict(transport=False, tiles=(4, 2, 1), pdl=False),
    "two-pass R8 C4 no-prefetch pdl": dict(transport=False, tiles=(8, 4, 0), pdl=True),
}


def _configurer(cfg):
    def f(ctx):
        if "transport" in cfg:
            ctx.set_transport(cfg["transport"])
            assert ctx.transport_config()[0] == int(cfg["transport"])
        if "tiles" in cfg:
            ctx.set_tiles(*cfg["tiles"])
        if "pdl" in cfg:
            ctx.set_pdl(cfg["pdl"])
    return f


@pytest.mark.parametrize("config", list(CONFIGS_512))
def test_registration_workload_512_nt32_matches_oracle(ref512, config):
    _compare(ref512, _configurer(CONFIGS_512[config]))


@pytest.mark.parametrize("pdl", [True, False])
def test_1024_grid_matches_oracle(ref1024, pdl):
    # 1024-point rows: R = 4 rows per CTA (512 threads) and C = 2 columns per column CTA are the
    # only valid tiles; the row kernels run without operand prefetch (two CTAs per SM)
    _compare(ref1024, _configurer(dict(tiles=(4, 2, 0), pdl=pdl)))


def test_1024_grid_has_no_cluster_path():
    from paper_1503_00757_gb300.binding import Context, RegError
    ctx = Context(1024, 1024, 2)
    assert ctx.transport_config()[:2] == (0, 0)
    with pytest.raises(RegError):
        ctx.set_transport(True)
    ctx.close()
