"""Batched registration (reg_solve_batch): every pair of a mixed-size,
mixed-setting batch solved concurrently must equal its standalone reg_solve
bit for bit (same kernels, same order, per-pair streams)."""
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


def _batch(nt=8):
    import torch
    rng = np.random.default_rng(4000)
    pairs = []
    for i, n in enumerate([64, 32, 64, 128, 32, 64]):
        mT, mR, _ = synth.ellipses_pair(n, 4000 + i, vmax=0.25 * 2 * np.pi * nt / n, kmax=min(16, n // 4))
        regnorm = int(rng.choice([1, 2]))
        gamma = [0.0, 1e-3, math.inf][int(rng.integers(3))]
        beta = [1e-2, 1e-3][int(rng.integers(2))]
        pairs.append(dict(mT=torch.tensor(mT, dtype=torch.float32, device="cuda"),
                          mR=torch.tensor(mR, dtype=torch.float32, device="cuda"),
                          v=torch.zeros(2, n, n, device="cuda"), nt=nt, regnorm=regnorm, beta=beta,
                          gamma=gamma, shear=0.0))
    return pairs


def test_batch_equals_sequential_solves():
    import torch
    from paper_1503_00757_gb300.binding import Context, default_opts, solve_batch
    pairs = _batch()
    opts = default_opts(tol=1e-2, maxit_newton=10)
    rc, stats = solve_batch(pairs, opts, nworkers=3, check=False)
    for p, st in zip(pairs, stats):
        n = p["mT"].shape[0]
        ctx = Context(n, n, p["nt"], regnorm=p["regnorm"], beta=p["beta"], gamma=p["gamma"])
        ctx.set_images(p["mT"], p["mR"])
        v = torch.zeros(2, n, n, device="cuda")
        ref = ctx.solve(v, opts, check=False)
        torch.cuda.synchronize()
        assert st["rc"] == ref["rc"]
        assert st["n_newton"] == ref["n_newton"] and st["n_mv"] == ref["n_mv"]
        assert torch.equal(p["v"], v)
        ctx.close()


def test_set_params_reuses_a_context():
    import torch
    from paper_1503_00757_gb300.binding import Context
    n = 64
    mT, mR, vs = synth.blobs_pair(n, 4100)
    v = torch.tensor(0.2 * vs, dtype=torch.float32, device="cuda")
    a = Context(n, n, 4, regnorm=2, beta=1e-3, gamma=1e-3)
    b = Context(n, n, 8, regnorm=1, beta=1e-2, gamma=math.inf)
    b.set_params(4, regnorm=2, beta=1e-3, gamma=1e-3)
    ga, gb = torch.empty_like(v), torch.empty_like(v)
    for c, g in ((a, ga), (b, gb)):
        c.set_images(torch.tensor(mT, dtype=torch.float32, device="cuda"),
                     torch.tensor(mR, dtype=torch.float32, device="cuda"))
        c.gradient(v, g)
    assert torch.equal(ga, gb)
