"""Pins for the oracle's FFT and spectral operators (CPU only).

Each check compares against something other than the oracle itself: the DFT
sum written out element by element, analytic derivatives of single Fourier
modes, the operator chain of Eq. (e:project-body-force) applied mode by mode,
and algebraic identities (Parseval, projector, skew-adjointness)."""
import cmath
import math

import numpy as np
import pytest

from oracle import fft as F
from oracle import spectral as S


def dft_sum(x):
    n = len(x)
    return np.array([sum(x[j] * cmath.exp(-2j * math.pi * j * k / n) for j in range(n)) for k in range(n)])


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32])
def test_fft_matches_dft_sum(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = F.fft(x)
    assert np.abs(X - dft_sum(x)).max() < 1e-12 * max(1, n)
    xi = F.fft(X, inverse=True) / n
    assert np.abs(xi - x).max() < 1e-14 * max(1, n)


def test_fft2_matches_dft_sum_and_axes():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((4, 8))
    X = F.fft2(x)
    ref = np.array([[sum(x[a, b] * cmath.exp(-2j * math.pi * (a * k1 / 4 + b * k2 / 8))
                         for a in range(4) for b in range(8)) for k2 in range(8)] for k1 in range(4)])
    assert np.abs(X - ref).max() < 1e-12
    assert np.abs(F.ifft2(X) - x).max() < 1e-14


def test_fft_parseval_delta_mode():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(64)
    X = F.fft(x)
    assert abs(np.sum(np.abs(X) ** 2) / 64 - np.sum(x ** 2)) < 1e-11
    d = np.zeros(16)
    d[0] = 1
    assert np.abs(F.fft(d) - 1).max() < 1e-15
    j = np.arange(16)
    e = np.exp(2j * np.pi * 5 * j / 16)
    E = F.fft(e)
    assert abs(E[5] - 16) < 1e-12 and np.abs(np.delete(E, 5)).max() < 1e-12


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        F.fft(np.zeros(12))


@pytest.mark.parametrize("k1,k2", [(1, 0), (0, 3), (2, -5), (-7, 4)])
def test_grad_div_lap_single_mode(k1, k2):
    n1, n2 = 16, 32
    X1, X2 = S.grid_coords(n1, n2)
    ph = k1 * X1 + k2 * X2
    f = np.cos(ph) + 0.5 * np.sin(ph)
    df = -np.sin(ph) + 0.5 * np.cos(ph)
    g = S.grad(f)
    assert np.abs(g[0] - k1 * df).max() < 1e-12
    assert np.abs(g[1] - k2 * df).max() < 1e-12
    assert np.abs(S.lap(f) + (k1 * k1 + k2 * k2) * f).max() < 1e-11
    u = np.stack([f, 2 * f])
    assert np.abs(S.div(u) - (k1 + 2 * k2) * df).max() < 1e-12
    for q, regnorm in [(1, S.H1), (2, S.H2)]:
        Av = S.apply_A(u, regnorm)
        assert np.abs(Av - (k1 * k1 + k2 * k2) ** q * u).max() < 1e-9 * (k1 * k1 + k2 * k2) ** q


def test_nyquist_readings():
    n = 16
    X1, X2 = S.grid_coords(n, n)
    f = np.cos(8 * X1)  # Nyquist mode along x^1
    assert np.abs(S.grad(f)).max() < 1e-13  # odd symbol: Nyquist set to 0
    assert np.abs(S.lap(f) + 64 * f).max() < 1e-11  # even symbol keeps |k| = n/2


def test_grad_is_minus_div_transpose():
    rng = np.random.default_rng(11)
    f = rng.standard_normal((16, 32))
    u = rng.standard_normal((2, 16, 32))
    assert abs(S.inner(S.grad(f), u) + S.inner(f, S.div(u))) < 1e-12 * np.sqrt(S.inner(f, f) * S.inner(u, u)) * 10


def _mode_vec(n1, n2, k1, k2, a):
    X1, X2 = S.grid_coords(n1, n2)
    c = np.cos(k1 * X1 + k2 * X2)
    return np.stack([a[0] * c, a[1] * c]), c


@pytest.mark.parametrize("regnorm", [S.H1, S.H2])
@pytest.mark.parametrize("beta_w", [0.0, 1e-3, 0.5, np.inf])
def test_projection_matches_elimination_chain(regnorm, beta_w):
    """K b = -grad M^-1 Lap^-1 div b + b with M = beta_v (beta_w(-Lap+I))^-1 + I
    for H1 (Eq. (e:project-body-force)); for H2 the same elimination with
    A = Lap^2 (Appendix A.1) gives M = beta_v (-Lap)(beta_w(-Lap+I))^-1 + I.
    Applied to cos modes, the chain is evaluated by hand: div -> -(k.a) sin,
    Lap^-1 -> /(-|k|^2), M^-1 -> /M, -grad -> ..."""
    n1, n2 = 16, 16
    beta_v = 1e-2
    for (k1, k2) in [(1, 2), (3, 0), (-2, 5), (4, 4)]:
        a = np.array([0.3, -1.1])
        b, c = _mode_vec(n1, n2, k1, k2, a)
        kk = k1 * k1 + k2 * k2
        ka = k1 * a[0] + k2 * a[1]
        if beta_w == 0.0:
            ref = b
        else:
            if np.isinf(beta_w):
                M = 1.0
            elif regnorm == S.H1:
                M = beta_v / (beta_w * (1 + kk)) + 1.0
            else:
                M = beta_v * kk / (beta_w * (1 + kk)) + 1.0
            # div b = -(k.a) sin(phase); Lap^-1 -> (k.a)/|k|^2 sin; M^-1; -grad of s sin = -s k cos
            s = ka / kk / M
            ref = b - s * np.stack([k1 * c, k2 * c])
        Kb = S.apply_K(b, regnorm, beta_v, beta_w)
        assert np.abs(Kb - ref).max() < 1e-12


def test_projection_eigenvalues_and_leray_identities():
    n = 32
    beta_v, beta_w = 1e-2, 1e-3
    K11, K12, K22 = S.projection_symbol(n, n, S.H1, beta_v, beta_w)
    K1o, K2o, KK = S.symbols(n, n)
    for i, j in [(1, 2), (5, 0), (3, 7)]:
        M = np.array([[K11[i, j], K12[i, j]], [K12[i, j], K22[i, j]]])
        k = np.array([K1o[i, j], K2o[i, j]])
        ev_par = k @ M @ k / (k @ k)
        kp = np.array([-k[1], k[0]])
        ev_perp = kp @ M @ kp / (kp @ kp)
        assert abs(ev_perp - 1) < 1e-14
        # eigenvalue along k: 1 - 1/M^ = beta_v / (beta_v + beta_w (1 + |k|^2))
        assert abs(ev_par - beta_v / (beta_v + beta_w * (1 + KK[i, j]))) < 1e-14
    rng = np.random.default_rng(5)
    b = rng.standard_normal((2, n, n))
    c = rng.standard_normal((2, n, n))
    P = S.apply_K(b, S.H1, beta_v, np.inf)
    assert np.abs(S.div(P)).max() < 1e-12
    assert np.abs(S.apply_K(P, S.H1, beta_v, np.inf) - P).max() < 1e-12
    for bw in [np.inf, beta_w]:
        assert abs(S.inner(S.apply_K(b, S.H1, beta_v, bw), c) - S.inner(b, S.apply_K(c, S.H1, beta_v, bw))) < 1e-11


def test_preconditioner_inverts_regularization():
    rng = np.random.default_rng(9)
    for regnorm in (S.H1, S.H2):
        v = rng.standard_normal((2, 16, 32))
        v -= v.mean(axis=(1, 2), keepdims=True)
        z = S.apply_precond(0.01 * S.apply_A(v, regnorm), regnorm, 0.01)
        assert np.abs(z - v).max() < 1e-10
        const = np.ones((2, 16, 32))
        assert np.abs(S.apply_precond(const, regnorm, 0.01) - 100.0).max() < 1e-10
