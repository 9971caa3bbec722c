"""Displacement field (Eq. (e:displacement)) and label-overlap measures (App. F) on the GPU
against the FP64 oracle.

Displacement: u_1 element by element (1e-5 relative L2) on a general velocity; a constant
velocity gives u_1 = v to FP32 rounding.  Label overlap: the transported smoothed template
labels element by element (1e-5); the thresholding is a discrete decision, so the measures
the library returns must equal the ones recomputed from its own transported field, and may
differ from the oracle's only through nodes within rounding of the 0.5 threshold.  A solved
registration raises the Dice coefficient above the unregistered one."""
import math

import numpy as np
import pytest

from oracle import measures as M
from oracle import transport as T
from paper_1503_00757_gb300 import synth

from .gpu_util import check, check_rel, make_ctx, to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00757_gb300.binding import lib
    lib()


@pytest.mark.parametrize("n,nt", [(64, 8), (128, 16), (256, 8)])
def test_displacement_matches_oracle(n, nt):
    import torch
    v = synth.velocity(n, n, max(2, n // 16), 0.25 * 2 * math.pi * nt / n, np.random.default_rng(n),
                       grad_fraction=0.4)
    ctx = make_ctx(n, n, nt)
    u = torch.empty(2, n, n, device="cuda")
    ctx.displacement(to_gpu(v), u)
    torch.cuda.synchronize()
    check_rel("displacement u_1", to_np(u), T.displacement_solve(v, nt), 1e-5)
    c = np.stack([np.full((n, n), 0.03), np.full((n, n), -0.02)])
    ctx.displacement(to_gpu(c), u)
    torch.cuda.synchronize()
    check("displacement, constant v (max abs)", np.abs(to_np(u) - c).max(), 1e-7)
    ctx.close()


def test_label_overlap_matches_oracle():
    import torch
    n, nt, seed, vmax = 128, 16, 3000, 0.2
    mT, mR, vs = synth.ellipses_pair(n, seed, vmax=vmax)
    LT, LR = synth.ellipse_labels(n, seed, vmax=vmax, label=1)
    ctx = make_ctx(n, n, nt, regnorm=1, beta=1e-3, gamma=math.inf)
    f = torch.empty(n, n, device="cuda")
    meas = ctx.label_overlap(to_gpu(vs), to_gpu(LT), to_gpu(LR), f)
    torch.cuda.synchronize()
    m1, LT1 = M.transported_labels(LT, vs, nt)
    fg = to_np(f)
    check_rel("transported labels", fg, m1, 1e-5)
    own = M.overlap(fg > 0.5, LR > 0.5)
    assert np.allclose(meas, own, rtol=0, atol=1e-12)
    ref = M.overlap(LT1, LR > 0.5)
    amb = np.count_nonzero(np.abs(m1 - 0.5) < 1e-5)
    nlab = np.count_nonzero(LR > 0.5)
    check("Dice vs oracle", abs(meas[1] - ref[1]), 2.0 * amb / nlab + 1e-12)
    # registering the pair improves the overlap of the labels
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    v = torch.zeros(2, n, n, device="cuda")
    st = ctx.solve(v)
    assert st["status"] == 0
    d0 = ctx.label_overlap(torch.zeros(2, n, n, device="cuda"), to_gpu(LT), to_gpu(LR))[1]
    d1 = ctx.label_overlap(v, to_gpu(LT), to_gpu(LR))[1]
    assert d1 > d0
    ctx.close()
