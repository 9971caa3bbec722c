"""FFT tile choices and their autotuner: every valid (rows per row
CTA, spectrum columns per column CTA, operand prefetch) gives the same
gradient and Hessian matvec bit for bit (each row and column transform is the
same code whatever the CTA holds; only FP64 reduction order may change J in
the last bits), and reg_autotune picks a valid choice that later contexts use."""
import math

import numpy as np
import pytest

from paper_1503_00757_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def valid_tiles(n1, n2):
    """The launch limits stated for reg_autotune, restated: [(R, C, P)]."""
    out = []
    R = 4
    while R <= n1:
        C = 2
        while C <= n2 // 2:
            # shared memory: staging plus two exchange buffers of L + L/8 entries per transform
            row_smem = (R * n2 + 2 * R * (n2 + n2 // 8)) * 8
            col_smem = (2 * C * n1 + 2 * C * (n1 + n1 // 8)) * 8
            ok = (n1 % R == 0 and 32 <= R * n2 // 8 <= 512 and row_smem <= 227 * 1024 and
                  (n2 // 2) % C == 0 and 32 <= C * n1 // 8 <= 256 and col_smem <= 227 * 1024)
            if ok:
                for P in ((0, 1) if n2 <= 512 else (0,)):
                    out.append((R, C, P))
            C *= 2
        R *= 2
    return out


@pytest.mark.parametrize("n1,n2", [(128, 128), (64, 256), (256, 64)])
def test_every_tile_choice_gives_identical_results(n1, n2):
    import torch
    from paper_1503_00757_gb300.binding import Context
    rng = np.random.default_rng(n1 + 7 * n2)
    mT = synth.gaussian_smooth(rng.random((n1, n2)), 0.15)
    mR = synth.gaussian_smooth(rng.random((n1, n2)), 0.15)
    v = 0.02 * np.stack([synth.gaussian_smooth(rng.standard_normal((n1, n2)), 0.3) for _ in range(2)])
    vt = np.stack([synth.gaussian_smooth(rng.standard_normal((n1, n2)), 0.3) for _ in range(2)])
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda").contiguous()
    stream = torch.cuda.Stream()  # a non-default stream: the captured-graph path
    ctx = Context(n1, n2, 8, regnorm=1, beta=1e-3, gamma=1e-3, stream=stream)
    ctx.set_transport(False)  # the row / column kernel pairs, whose tiles are under test
    mTd, mRd, vd, vtd = dev(mT), dev(mR), dev(v), dev(vt)
    g0, h0 = torch.empty(2, n1, n2, device="cuda"), torch.empty(2, n1, n2, device="cuda")
    torch.cuda.synchronize()
    ctx.set_images(mTd, mRd)
    ctx.set_tiles(0, 0, 0)
    J0 = ctx.gradient(vd, g0)
    ctx.hessian_matvec(vtd, h0)
    cands = valid_tiles(n1, n2)
    assert len(cands) >= 2
    for R, C, P in cands:
        ctx.set_tiles(R, C, P)
        assert ctx.tile_config()[:3] == (R, C, P)
        ctx.set_pdl(R % 8 == 0)  # both launch modes give the same results too
        g, h = torch.empty_like(g0), torch.empty_like(h0)
        torch.cuda.synchronize()
        J = ctx.gradient(vd, g)
        ctx.hessian_matvec(vtd, h)
        stream.synchronize()
        assert torch.equal(g, g0), (R, C, P)
        assert torch.equal(h, h0), (R, C, P)
        assert abs(J - J0) <= 1e-12 * abs(J0)
    ctx.close()


def test_invalid_tiles_rejected():
    from paper_1503_00757_gb300.binding import Context, RegError
    ctx = Context(128, 128, 4)
    for R, C, P in [(6, 4, 0), (256, 4, 0), (4, 3, 0), (4, 128, 0), (2, 4, 0), (4, 4, 2)]:
        with pytest.raises(RegError):
            ctx.set_tiles(R, C, P)
    ctx.close()
    big = Context(64, 1024, 4)
    with pytest.raises(RegError):
        big.set_tiles(4, 4, 1)  # no prefetch variant for 1024-point rows
    big.close()
    ctx.close()


def test_autotune_picks_a_valid_pair_used_by_later_contexts():
    from paper_1503_00757_gb300.binding import Context, autotune
    for conc in (1, 3):
        R, C, P, D, ms = autotune(128, 256, nt=4, concurrency=conc, force=True)
        assert (R, C, P) in valid_tiles(128, 256) and D in (0, 1)
        assert ms > 0.0
        ctx = Context(128, 256, 4)
        assert ctx.tile_config() == (R, C, P, D)
        ctx.close()
        R2, C2, P2, D2, ms2 = autotune(128, 256, nt=4)
        assert (R2, C2, P2, D2) == (R, C, P, D) and ms2 < 0.0  # cached
