"""What the trained warm-start network gains over the plain zero start.

The committed weights (trained on solver-generated targets, 256^2 pairs of the learned-start
workload) and their calibrated output scale are loaded; 32 held-out seeded pairs (seeds
6 000 000 + i, disjoint from the training and calibration seeds) are registered twice through
the batch executor: from v = 0 and from the network's prediction.  The zero-start solve stays
the judge: every warm-started solve must reach the same stopping test ||g|| <= 1e-2 ||g(0)||
(g_ref = g(0) for both), with status REG_OK, and the warm starts must take fewer Gauss-Newton
matvecs in total (the solver's dominant cost) and fewer Newton iterations on average."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_1503_00757_gb300", "weights", "warmstart_n256.npy")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_trained_network_cuts_matvecs_at_the_same_tolerance():
    import torch
    from paper_1503_00757_gb300 import warmstart as ws
    from paper_1503_00757_gb300.binding import Executor, Net, default_opts
    assert os.path.exists(WEIGHTS)
    scale = json.load(open(os.path.splitext(WEIGHTS)[0] + ".json"))["output_scale"]
    x = ws.make_images(256, range(ws.TEST_SEED, ws.TEST_SEED + 32))
    ex = Executor(8)
    net = Net(256, 256, 8)
    net.set_params(torch.from_numpy(np.load(WEIGHTS).astype(np.float32)).cuda())
    net.set_output_scale(scale)
    opts0 = default_opts(tol=1e-2)
    _, st0, _ = ws.solve_all(x, ex, opts0)
    v0 = ws.predict(net, x, 8)
    _, st1, _ = ws.solve_all(x, ex, default_opts(tol=1e-2, warm_start=1), v0=v0)
    net.close()
    ex.close()
    for a, b in zip(st0, st1):
        assert a["rc"] == 0 and a["gnorm_rel"] <= 1e-2
        assert b["rc"] == 0 and b["gnorm_rel"] <= 1e-2  # same stopping test, relative to g(0)
    mv0 = sum(s["n_mv"] for s in st0)
    mv1 = sum(s["n_mv"] for s in st1)
    nw0 = np.mean([s["n_newton"] for s in st0])
    nw1 = np.mean([s["n_newton"] for s in st1])
    print(f"zero start: {mv0 / len(st0):.1f} matvecs, {nw0:.2f} Newton; "
          f"warm start: {mv1 / len(st1):.1f} matvecs, {nw1:.2f} Newton")
    assert mv1 < 0.95 * mv0
    assert nw1 <= nw0
