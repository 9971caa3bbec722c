"""Own radix-2 fast Fourier transform in FP64 (oracle; test infrastructure only).

The paper discretizes space with a pseudospectral Fourier basis (Sec. 4,
"Numerics").  The oracle does not rely on a library FFT for this: it runs a
textbook iterative Cooley-Tukey decimation-in-time transform (bit-reversal
permutation, then log2(n) butterfly sweeps), vectorized over all other axes.

Convention (unnormalized forward, 1/n on the inverse):

    X[k] = sum_j x[j] exp(-2 pi i j k / n),     x[j] = (1/n) sum_k X[k] exp(+2 pi i j k / n)

Pinned in ``tests/test_oracle_fft.py`` against the O(n^2) DFT sum written out
element by element, Parseval's identity, delta and single-mode transforms.
"""
import numpy as np


def _bit_reversal(n):
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft(x, axis=-1, inverse=False):
    """Unnormalized 1-D DFT (or its conjugate-sign counterpart) along ``axis``."""
    y = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = y.shape[-1]
    if n < 1 or (n & (n - 1)) != 0:
        raise ValueError(f"length {n} is not a power of two")
    y = y[..., _bit_reversal(n)]
    lead = y.shape[:-1]
    sign = 1.0 if inverse else -1.0
    half = 1
    while half < n:
        # butterflies combining pairs of length-`half` transforms into length 2*half
        w = np.exp(sign * 1j * np.pi * np.arange(half) / half)
        y = y.reshape(lead + (n // (2 * half), 2, half))
        a = y[..., 0, :]
        b = y[..., 1, :] * w
        y = np.stack([a + b, a - b], axis=-2).reshape(lead + (n,))
        half *= 2
    return np.moveaxis(y, -1, axis)


def fft2(x):
    """2-D DFT over the last two axes (rows = x^1 index, columns = x^2 index)."""
    return fft(fft(x, axis=-2), axis=-1)


def ifft2(X):
    """Inverse 2-D DFT over the last two axes, including the 1/(n1 n2) factor."""
    n1, n2 = X.shape[-2], X.shape[-1]
    return fft(fft(X, axis=-2, inverse=True), axis=-1, inverse=True) / (n1 * n2)
