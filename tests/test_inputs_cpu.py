"""CPU checks of the seeded synthetic inputs (paper_1503_00757_gb300/synth.py) against the
recipe they implement, measured with numpy's FFT (an instrument independent of both the
generator and the oracle): the velocities are band-limited, scaled to the stated maximum
norm, and divergence-free or carry the stated gradient fraction; images are rescaled to
[0, 1], the reference image is a warp of the template by v*, and every input is a
deterministic function of its seed."""
import math
import os
import sys

import numpy as np
import pytest

from paper_1503_00757_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _wavenumbers(n1, n2):
    k1 = np.fft.fftfreq(n1, 1.0 / n1)
    k2 = np.fft.fftfreq(n2, 1.0 / n2)
    return np.meshgrid(k1, k2, indexing="ij")


def _helmholtz(v):
    """(divergence-free part, curl-free part) of a periodic vector field by Fourier projection."""
    n1, n2 = v.shape[1:]
    K1, K2 = _wavenumbers(n1, n2)
    kk = K1 ** 2 + K2 ** 2
    kk[0, 0] = 1.0
    V1, V2 = np.fft.fft2(v[0]), np.fft.fft2(v[1])
    d = (K1 * V1 + K2 * V2) / kk
    G1, G2 = K1 * d, K2 * d
    grad = np.stack([np.real(np.fft.ifft2(G1)), np.real(np.fft.ifft2(G2))])
    return v - grad, grad


@pytest.mark.parametrize("n1,n2,kmax", [(64, 64, 4), (64, 128, 16), (128, 64, 8)])
def test_velocity_is_divergence_free_band_limited_and_scaled(n1, n2, kmax):
    v = synth.velocity(n1, n2, kmax, 0.37, np.random.default_rng(11))
    assert v.shape == (2, n1, n2)
    assert abs(np.sqrt(v[0] ** 2 + v[1] ** 2).max() - 0.37) < 1e-14
    K1, K2 = _wavenumbers(n1, n2)
    V1, V2 = np.fft.fft2(v[0]), np.fft.fft2(v[1])
    div = np.abs(K1 * V1 + K2 * V2)
    assert div.max() < 1e-12 * np.abs(V1).max()
    outside = K1 ** 2 + K2 ** 2 > kmax * kmax
    energy = np.abs(V1) ** 2 + np.abs(V2) ** 2
    assert energy[outside].sum() < 1e-24 * energy.sum()
    assert energy[0, 0] < 1e-24 * energy.sum()  # no mean flow


def test_velocity_gradient_fraction():
    v = synth.velocity(128, 128, 8, 0.8, np.random.default_rng(5), grad_fraction=0.3)
    div_free, curl_free = _helmholtz(v)
    rms = lambda a: np.sqrt(np.mean(a ** 2))
    assert abs(rms(curl_free) / rms(div_free) - 0.3) < 1e-10


def test_velocity_rejects_modes_at_nyquist():
    with pytest.raises(ValueError):
        synth.velocity(32, 32, 16, 0.1, np.random.default_rng(0))


@pytest.mark.parametrize("make", [
    lambda s: synth.blobs_pair(64, s),
    lambda s: synth.ellipses_pair(64, s, vmax=0.2, kmax=8),
    lambda s: synth.labels_pair(64, s, kmax=8),
])
def test_pairs_are_rescaled_and_deterministic(make):
    mT, mR, v = make(1234)
    assert mT.shape == mR.shape == (64, 64) and v.shape == (2, 64, 64)
    assert mT.min() == 0.0 and mT.max() == 1.0
    assert -0.1 < mR.min() and mR.max() < 1.1
    mT2, mR2, v2 = make(1234)
    assert np.array_equal(mT, mT2) and np.array_equal(mR, mR2) and np.array_equal(v, v2)
    mT3, _, v3 = make(1235)
    assert not np.array_equal(v, v3)


def test_reference_is_a_warp_of_the_template():
    # with a vanishing displacement the reference equals the template; with the stated
    # one it differs, by about |grad m_T| |v*| to first order
    mT, mR, _ = synth.blobs_pair(64, 7, vmax=1e-9)
    assert np.abs(mR - mT).max() < 1e-7
    mT, mR, v = synth.ellipses_pair(128, 7, vmax=0.05, kmax=8)
    h = 2 * math.pi / 128
    g1 = (np.roll(mT, -1, 0) - np.roll(mT, 1, 0)) / (2 * h)
    g2 = (np.roll(mT, -1, 1) - np.roll(mT, 1, 1)) / (2 * h)
    first_order = -(g1 * v[0] + g2 * v[1])
    diff = mR - mT
    assert np.abs(diff).max() > 0.05
    assert np.linalg.norm(diff - first_order) < 0.35 * np.linalg.norm(diff)


@pytest.mark.parametrize("k1,k2", [(0, 3), (5, -2), (7, 7)])
def test_gaussian_smooth_symbol(k1, k2):
    X1, X2 = synth.coords(32, 64)
    f = np.cos(k1 * X1 + k2 * X2)
    sigma = 0.2
    out = synth.gaussian_smooth(f, sigma)
    assert np.abs(out - math.exp(-0.5 * sigma * sigma * (k1 * k1 + k2 * k2)) * f).max() < 1e-13


def test_image_batch_matches_single_pairs():
    jobs = [(64, 6000000, 0.098), (64, 6000001, 0.098)]
    imgs = synth.ellipses_images(jobs, workers=1)
    for (n, seed, vmax), (mT, mR) in zip(jobs, imgs):
        eT, eR, _ = synth.ellipses_pair(n, seed, vmax=vmax, kmax=min(16, n // 4))
        assert mT.dtype == np.float32 and np.array_equal(mT, eT.astype(np.float32))
        assert np.array_equal(mR, eR.astype(np.float32))


def test_registration_workload_cfl():
    sys.path.insert(0, ROOT)
    import bench
    # CFL number max|v| h_t / h_x with h_t = 1/nt, h_x = 2 pi / n: 0.25 at 512^2 and nt = 32
    cfl = bench.VMAX / bench.NT / (2 * math.pi / bench.N_GRID)
    assert abs(cfl - 0.25) < 0.001
    v = synth.ellipses_pair(64, bench.SEED, vmax=bench.VMAX)[2]
    assert abs(np.sqrt(v[0] ** 2 + v[1] ** 2).max() - bench.VMAX) < 1e-14
