"""Pins for the warm-start network oracle: the convolution against its
definition written as explicit index loops, the backward pass against finite
differences of the loss, and the divergence-free output."""
import numpy as np

from oracle import cnn
from oracle import spectral as S


def conv_loops(a, W, b):
    B, C, H, Wd = a.shape
    O = W.shape[0]
    out = np.zeros((B, O, H, Wd))
    for bb in range(B):
        for o in range(O):
            for y in range(H):
                for x in range(Wd):
                    s = b[o]
                    for c in range(C):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                s += W[o, c, dy + 1, dx + 1] * a[bb, c, (y + dy) % H, (x + dx) % Wd]
                    out[bb, o, y, x] = s
    return out


def test_conv_matches_index_loops():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 3, 5, 6))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    assert np.abs(cnn.conv3x3(a, W, b) - conv_loops(a, W, b)).max() < 1e-12


def test_conv_backward_is_adjoint():
    """<conv(a), dz> = <a, conv^T dz> (bias 0) and dW from the loop definition."""
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 3, 6, 5))
    W = rng.standard_normal((4, 3, 3, 3))
    dz = rng.standard_normal((2, 4, 6, 5))
    da, dW, db = cnn.conv3x3_backward(a, W, dz)
    lhs = np.sum(cnn.conv3x3(a, W, np.zeros(4)) * dz)
    assert abs(lhs - np.sum(a * da)) < 1e-10 * abs(lhs)
    eps = 1e-6
    for (o, c, i, j) in [(0, 0, 0, 0), (3, 2, 1, 2), (1, 1, 2, 1)]:
        Wp = W.copy()
        Wp[o, c, i, j] += eps
        fd = (np.sum(cnn.conv3x3(a, Wp, np.zeros(4)) * dz) - lhs) / eps
        assert abs(fd - dW[o, c, i, j]) < 1e-5 * max(1, abs(fd))
    assert np.abs(db - dz.sum(axis=(0, 2, 3))).max() < 1e-12


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    ch = (2, 3, 3, 2)
    params = cnn.init_params(3, ch)
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    x = rng.standard_normal((2, 2, 8, 8))
    t = cnn.leray(rng.standard_normal((2, 2, 8, 8)))
    loss, grads = cnn.loss_and_grads(params, x, t)
    eps = 1e-6
    for l, (W, b) in enumerate(params):
        for idx in [(0, 0, 1, 1), (W.shape[0] - 1, W.shape[1] - 1, 2, 0)]:
            Wp = W.copy()
            Wp[idx] += eps
            pp = list(params)
            pp[l] = (Wp, b)
            Wm = W.copy()
            Wm[idx] -= eps
            pm = list(params)
            pm[l] = (Wm, b)
            fd = (cnn.loss_and_grads(pp, x, t)[0] - cnn.loss_and_grads(pm, x, t)[0]) / (2 * eps)
            assert abs(fd - grads[l][0][idx]) < 1e-6 * max(1e-3, abs(fd)) + 1e-10
        bp = b.copy()
        bp[0] += eps
        pp = list(params)
        pp[l] = (W, bp)
        bm = b.copy()
        bm[0] -= eps
        pm = list(params)
        pm[l] = (W, bm)
        fd = (cnn.loss_and_grads(pp, x, t)[0] - cnn.loss_and_grads(pm, x, t)[0]) / (2 * eps)
        assert abs(fd - grads[l][1][0]) < 1e-6 * max(1e-3, abs(fd)) + 1e-10


def test_prediction_is_divergence_free():
    params = cnn.init_params(4, (2, 4, 2))
    x = np.random.default_rng(5).standard_normal((1, 2, 16, 16))
    v = cnn.predict(params, x)
    assert np.abs(S.div(v[0])).max() < 1e-12
