"""CPU checks of the warm-start pipeline's host logic: the flat parameter layout that
reg_net_set_params reads, the He initialisation, the output-scale selection, and the
summary statistics (no GPU: the network and the solver are replaced by fakes where needed)."""
import numpy as np
import pytest

from paper_1503_00757_gb300 import warmstart as ws
from paper_1503_00757_gb300.binding import flatten_params, unflatten_params


def test_flat_layout_round_trip_and_size():
    params = ws.he_init(3)
    flat = flatten_params(params)
    # per layer W (Cout, Cin, 3, 3) then b (Cout)
    want = sum(cout * cin * 9 + cout for cin, cout in zip(ws.CHANNELS[:-1], ws.CHANNELS[1:]))
    assert flat.size == want == 2 * 32 * 9 + 32 + 6 * (32 * 32 * 9 + 32) + 32 * 2 * 9 + 2
    back = unflatten_params(flat, ws.CHANNELS)
    assert len(back) == len(params) == 8
    for (W, b), (W2, b2) in zip(params, back):
        assert np.array_equal(W, W2) and np.array_equal(b, b2)
    # the first weight of layer 2 sits right after layer 1's W and b
    assert flat[2 * 32 * 9 + 32] == params[1][0][0, 0, 0, 0]


def test_he_init_variance_and_determinism():
    params = ws.he_init(7)
    for (W, b), cin in zip(params, ws.CHANNELS[:-1]):
        assert not b.any()
        var = 2.0 / (9.0 * cin)
        # sample variance within 5 standard errors of a Gaussian's (2 var^2 / (n - 1))
        se = var * np.sqrt(2.0 / (W.size - 1))
        assert abs(W.var() - var) < 5 * se
    again = ws.he_init(7)
    assert all(np.array_equal(a[0], c[0]) for a, c in zip(params, again))
    assert not np.array_equal(params[0][0], ws.he_init(8)[0][0])


def test_summarize():
    st = [{"rc": 0, "n_newton": 4, "n_mv": 40, "gnorm_rel": 0.008},
          {"rc": 10, "n_newton": 6, "n_mv": 50, "gnorm_rel": 0.02}]
    s = ws.summarize(st, 2.0)
    assert s["pairs"] == 2 and s["converged"] == 1
    assert s["newton_mean"] == 5.0 and s["matvec_mean"] == 45.0
    assert s["gnorm_rel_max"] == 0.02 and s["registrations_per_s"] == 1.0


@pytest.fixture(scope="module")
def built_library():
    """calibrate_scale builds its solver options through the C library (no CUDA call)."""
    import os
    from paper_1503_00757_gb300 import build as b
    if not os.path.exists(b.LIB_PATH):
        b.build()


class _FakeNet:
    def __init__(self):
        self.scale = 1.0
        self.history = []

    def set_output_scale(self, s):
        self.scale = s
        self.history.append(s)


@pytest.mark.parametrize("cost,want", [
    ({0.5: 50, 0.6: 44, 0.7: 43, 0.8: 45, 1.0: 51}, 0.7),
    ({0.5: 50, 0.6: 43, 0.7: 43, 0.8: 45}, 0.7),     # a tie goes to the larger scale
    ({0.6: 40, 0.7: 41}, 0.6),
])
def test_calibrate_scale_picks_fewest_matvecs(built_library, monkeypatch, cost, want):
    net = _FakeNet()
    monkeypatch.setattr(ws, "predict", lambda n, images, batch: n.scale)

    def fake_solve_all(images, executor, opts, v0=None, chunk=64):
        assert opts.warm_start == 1
        n_mv = cost[v0]
        return None, [{"rc": 0, "n_newton": 4, "n_mv": n_mv, "gnorm_rel": 0.009}] * 3, 1.0

    monkeypatch.setattr(ws, "solve_all", fake_solve_all)
    best, table = ws.calibrate_scale(net, images=None, executor=None, scales=list(cost), batch=8)
    assert best == want
    assert set(table) == set(cost) and all(table[s]["matvec_mean"] == cost[s] for s in cost)
    assert net.scale == 1.0  # restored after the sweep
