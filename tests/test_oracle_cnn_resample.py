"""Pins for the oracle's grid transfer of the doubled-grid warm start (restrict2, prolong2):
single Fourier modes, whose images under both maps are closed forms (full weighting multiplies
cos(k . x) by (1 + cos(k1 h)) / 2 * (1 + cos(k2 h)) / 2 at the coarse nodes, h the fine spacing;
bilinear interpolation keeps the coarse nodes and puts the mode times cos(k h_c / 2) at edge
midpoints and times cos(k1 h_c / 2) cos(k2 h_c / 2) at cell centres), constants, and the
composition's divergence-free output."""
import numpy as np

from oracle import cnn
from oracle import spectral as S


def _mode(n, k1, k2, phase=0.3):
    x = np.arange(n) * (2 * np.pi / n)
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    return np.cos(k1 * X1 + k2 * X2 + phase), X1, X2


def test_restrict2_full_weighting_symbol():
    n = 64
    h = 2 * np.pi / n
    for k1, k2 in [(1, 0), (3, -5), (7, 11)]:
        f, _, _ = _mode(n, k1, k2)
        c, _, _ = _mode(n // 2, k1, k2)
        sym = 0.5 * (1 + np.cos(k1 * h)) * 0.5 * (1 + np.cos(k2 * h))
        assert np.abs(cnn.restrict2(f) - sym * c).max() < 1e-13


def test_prolong2_nodes_midpoints_centres():
    n = 32
    hc = 2 * np.pi / n
    for k1, k2 in [(1, 2), (4, -3)]:
        c, _, _ = _mode(n, k1, k2)
        f, _, _ = _mode(2 * n, k1, k2)
        p = cnn.prolong2(c)
        assert np.array_equal(p[::2, ::2], c)
        # edge midpoints along x2 (y even, x odd): the mode times cos(k2 hc / 2)
        assert np.abs(p[::2, 1::2] - np.cos(k2 * hc / 2) * f[::2, 1::2]).max() < 1e-13
        assert np.abs(p[1::2, ::2] - np.cos(k1 * hc / 2) * f[1::2, ::2]).max() < 1e-13
        # cell centres: the average of the four corners
        cc = 0.5 * (np.cos((k1 + k2) * hc / 2) + np.cos((k1 - k2) * hc / 2))
        assert np.abs(p[1::2, 1::2] - cc * f[1::2, 1::2]).max() < 1e-13


def test_constants_and_batch_axes():
    u = np.full((2, 3, 16, 16), 1.7)
    assert np.allclose(cnn.restrict2(u), 1.7, atol=1e-15) and cnn.restrict2(u).shape == (2, 3, 8, 8)
    assert np.allclose(cnn.prolong2(u), 1.7, atol=1e-15) and cnn.prolong2(u).shape == (2, 3, 32, 32)


def test_predict_fine_is_divergence_free_and_scaled():
    rng = np.random.default_rng(0)
    params = cnn.init_params(3, channels=(2, 4, 2))
    x = rng.random((1, 2, 64, 64))
    v1 = cnn.predict_fine(params, x)
    v2 = cnn.predict_fine(params, x, scale=0.5)
    assert v1.shape == (1, 2, 64, 64)
    assert np.abs(S.div(v1[0])).max() < 1e-10 * max(np.abs(v1).max(), 1e-30)
    assert np.allclose(v2, 0.5 * v1, rtol=0, atol=1e-15)
