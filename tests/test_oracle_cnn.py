"""Pins for the warm-start network oracle: the (dilated) convolution against
its definition written as explicit index loops, the backward pass against
finite differences of the loss, the output low-pass on single Fourier modes,
and the divergence-free output."""
import numpy as np

from oracle import cnn
from oracle import spectral as S


def conv_loops(a, W, b, d=1):
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
                                s += W[o, c, dy + 1, dx + 1] * a[bb, c, (y + d * dy) % H, (x + d * dx) % Wd]
                    out[bb, o, y, x] = s
    return out


def test_conv_matches_index_loops():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 3, 5, 6))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    assert np.abs(cnn.conv3x3(a, W, b) - conv_loops(a, W, b)).max() < 1e-12


def test_dilated_conv_matches_index_loops():
    rng = np.random.default_rng(7)
    a = rng.standard_normal((1, 2, 12, 10))
    W = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    for d in (2, 3, 5):
        assert np.abs(cnn.conv3x3(a, W, b, d) - conv_loops(a, W, b, d)).max() < 1e-12


def test_dilated_conv_backward_is_adjoint():
    rng = np.random.default_rng(8)
    a = rng.standard_normal((2, 3, 12, 16))
    W = rng.standard_normal((2, 3, 3, 3))
    dz = rng.standard_normal((2, 2, 12, 16))
    d = 3
    da, dW, _ = cnn.conv3x3_backward(a, W, dz, d)
    lhs = np.sum(cnn.conv3x3(a, W, np.zeros(2), d) * dz)
    assert abs(lhs - np.sum(a * da)) < 1e-10 * abs(lhs)
    ref = np.zeros_like(W)
    for o in range(2):
        for c in range(3):
            for i in range(3):
                for j in range(3):
                    E = np.zeros_like(W)
                    E[o, c, i, j] = 1.0
                    ref[o, c, i, j] = np.sum(conv_loops(a, E, np.zeros(2), d) * dz)
    assert np.abs(dW - ref).max() < 1e-10 * np.abs(ref).max()


def test_dilation_schedule():
    assert cnn.dilations(256, 256) == [1, 2, 4, 8, 8, 4, 2, 1]
    assert cnn.dilations(64, 64) == [1, 2, 2, 2, 2, 2, 2, 1]
    assert cnn.dilations(32, 32) == [1] * 8
    assert cnn.dilations(16, 256) == [1, 2, 2, 2, 2, 2, 2, 1]


def test_output_lowpass_on_single_modes():
    """cos(k.x) is an eigenfunction of G with eigenvalue exp(-sigma^2 |k|^2 / 2),
    the Nyquist mode included (|k_Nyq| = n/2)."""
    H, W = 16, 32
    x1, x2 = S.grid_coords(H, W)
    s = cnn.gauss_sigma(H, W)
    assert abs(s - 2 * 2 * np.pi / 32) < 1e-15
    for k1, k2 in [(0, 0), (1, 0), (3, -5), (8, 0), (0, 16), (8, 16), (-7, 11)]:
        u = np.cos(k1 * x1 + k2 * x2)[None, None]
        lam = np.exp(-0.5 * s * s * (k1 * k1 + k2 * k2))
        assert np.abs(cnn.gauss(u) - lam * u).max() < 1e-12


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


def test_dilated_network_gradients_match_finite_differences():
    """Same check on a grid where the middle layers are dilated (d = 2)."""
    rng = np.random.default_rng(3)
    ch = (2, 3, 3, 2)
    assert cnn.dilations(16, 64, 3) == [1, 2, 2]
    params = cnn.init_params(4, ch)
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    x = rng.standard_normal((1, 2, 16, 64))
    t = cnn.leray(rng.standard_normal((1, 2, 16, 64)))
    loss, grads = cnn.loss_and_grads(params, x, t)
    eps = 1e-6
    for l, (W, b) in enumerate(params):
        idx = (W.shape[0] - 1, 0, 0, 2)
        Wp = W.copy()
        Wp[idx] += eps
        Wm = W.copy()
        Wm[idx] -= eps
        pp, pm = list(params), list(params)
        pp[l], pm[l] = (Wp, b), (Wm, b)
        fd = (cnn.loss_and_grads(pp, x, t)[0] - cnn.loss_and_grads(pm, x, t)[0]) / (2 * eps)
        assert abs(fd - grads[l][0][idx]) < 1e-6 * max(1e-3, abs(fd)) + 1e-10


def test_prediction_is_divergence_free():
    params = cnn.init_params(4, (2, 4, 2))
    x = np.random.default_rng(5).standard_normal((1, 2, 16, 16))
    v = cnn.predict(params, x)
    assert np.abs(S.div(v[0])).max() < 1e-12
