"""Pseudospectral differential operators on the periodic grid (oracle; test
infrastructure only).

Domain and grid.  The paper's domain is Omega = (-pi, pi)^2 with periodic
boundary conditions (notation, Sec. 1.5).  On a periodic grid this is the
same as [0, 2 pi)^2; node (i, j) sits at x = (2 pi i / n1, 2 pi j / n2).  Arrays
are indexed [i, j]: axis 0 is x^1 ("rows"), axis 1 is x^2 ("columns").

Quadrature.  Inner products use the trapezoidal rule the paper names in Sec. 4,
which on a periodic grid is <f, g> = h1 h2 sum f g with h = 2 pi / n.

Fourier symbols (readings the paper leaves open, stated once here):
  * integer wavenumbers k in {-n/2, ..., n/2 - 1} per axis;
  * odd-order operators (gradient, divergence) use k~ = k with the Nyquist
    entry set to 0, so the spectral gradient matrix is real and exactly
    skew-symmetric (grad^T = -div under <.,.>);
  * even-order operators (the regularization operator A, the H1 operator on
    the mass source) use the full |k|^2 with |k_Nyquist| = n/2.

Operators:
  * A[v] = -Lap v (H1), Lap^2 v (H2) or -Lap^3 v (H3), Eq. (e:var-reg-v) and App. A.1:
    symbol |k|^2, |k|^4 or |k|^6.
  * K[b] = -grad M^-1 Lap^-1 div b + b, M = beta_v (beta_w(-Lap + I))^-1 + I,
    Eq. (e:project-body-force), derived in Appendix A.1 (Eqs. (e:mass-source),
    (e:pressure-elimination-relaxed-ic), (e:derive-control-eq-elim)).  Taking
    the divergence of the control equation with the discrete symbols above
    gives p^ = i k~.b^ / (|k~|^2 + beta_v A^(k) / (beta_w (1 + |k|^2))), hence the
    2x2 Fourier multiplier
        K^(k) = I - k~ k~^T / (|k~|^2 + beta_v A^(k) / (beta_w (1 + |k|^2))),
    and K^ = I where k~ = 0.  For H1 and |k~| = |k| this is exactly
    I - k k^T / (|k|^2 M^(k)) with M^ = 1 + beta_v / (beta_w (1 + |k|^2)).
    The same derivation with A = Lap^2 is the H2 case the paper says follows
    by "the same arguments" (Appendix A.1).  Limits: beta_w = +inf (w = 0)
    gives the Leray projector I - k~k~^T/|k~|^2; beta_w = 0 (gamma = 0)
    gives K = I.
  * Preconditioner (beta_v A)^-1 (Appendix E, "Preconditioning"), with the
    kernel of A modified so that it is invertible: the symbol at k = 0 is
    set to 1, i.e. z^(0) = r^(0) / beta_v.
"""
import numpy as np

from .fft import fft2, ifft2

H1 = 1
H2 = 2
H3 = 3


def spacing(shape):
    n1, n2 = shape[-2], shape[-1]
    return 2.0 * np.pi / n1, 2.0 * np.pi / n2


def grid_coords(n1, n2):
    """Node coordinates x^1 (varies along axis 0) and x^2 (along axis 1)."""
    x1 = 2.0 * np.pi * np.arange(n1) / n1
    x2 = 2.0 * np.pi * np.arange(n2) / n2
    return np.meshgrid(x1, x2, indexing="ij")


def inner(f, g):
    """Trapezoidal-rule L2 inner product; sums over every component."""
    h1, h2 = spacing(np.shape(f))
    return float(h1 * h2 * np.sum(np.asarray(f, dtype=np.float64) * np.asarray(g, dtype=np.float64)))


def norm(f):
    return float(np.sqrt(inner(f, f)))


def wavenumbers(n):
    """(k, k_odd, k_even): signed integer wavenumbers in DFT order; the
    Nyquist entry is 0 in k_odd and n/2 in k_even."""
    k = np.concatenate([np.arange(0, n // 2), np.arange(-n // 2, 0)]).astype(np.float64)
    k_odd = k.copy()
    k_odd[n // 2] = 0.0
    k_even = k.copy()
    k_even[n // 2] = n / 2.0
    return k, k_odd, k_even


def symbols(n1, n2):
    """2-D arrays (k1~, k2~, |k|^2) on the full n1 x n2 spectrum."""
    _, k1o, k1e = wavenumbers(n1)
    _, k2o, k2e = wavenumbers(n2)
    K1o, K2o = np.meshgrid(k1o, k2o, indexing="ij")
    K1e, K2e = np.meshgrid(k1e, k2e, indexing="ij")
    return K1o, K2o, K1e ** 2 + K2e ** 2


def _real(Z):
    return np.real(Z)


def grad(f):
    """Spectral gradient of a scalar field: returns array (2, n1, n2)."""
    n1, n2 = f.shape
    K1o, K2o, _ = symbols(n1, n2)
    F = fft2(f)
    return np.stack([_real(ifft2(1j * K1o * F)), _real(ifft2(1j * K2o * F))])


def div(u):
    """Spectral divergence of a vector field u (2, n1, n2)."""
    n1, n2 = u.shape[-2:]
    K1o, K2o, _ = symbols(n1, n2)
    return _real(ifft2(1j * K1o * fft2(u[0]) + 1j * K2o * fft2(u[1])))


def lap(f):
    """Spectral Laplacian (even symbol -|k|^2) of a scalar field."""
    n1, n2 = f.shape
    _, _, KK = symbols(n1, n2)
    return _real(ifft2(-KK * fft2(f)))


def reg_symbol(n1, n2, regnorm):
    """A^(k): |k|^2 for the H1 seminorm, |k|^4 for the H2 seminorm (Eq. (e:var-reg-v)), |k|^6
    for the H3 seminorm (the triharmonic control equation App. A.1 names as the next choice)."""
    _, _, KK = symbols(n1, n2)
    if regnorm == H1:
        return KK
    if regnorm == H2:
        return KK ** 2
    if regnorm == H3:
        return KK ** 3
    raise ValueError("regnorm must be 1 (H1), 2 (H2) or 3 (H3)")


def apply_A(v, regnorm):
    """First (= second) variation of the quadratic seminorm, Eq. (e:var-reg-v),
    applied componentwise to a vector field (2, n1, n2)."""
    n1, n2 = v.shape[-2:]
    Ah = reg_symbol(n1, n2, regnorm)
    return np.stack([_real(ifft2(Ah * fft2(v[c]))) for c in range(2)])


def apply_W(w):
    """(-Lap + I) w: first variation of the H1 norm on the mass source, Eq. (e:reg-w)."""
    n1, n2 = w.shape
    _, _, KK = symbols(n1, n2)
    return _real(ifft2((1.0 + KK) * fft2(w)))


def projection_symbol(n1, n2, regnorm, beta_v, beta_w):
    """2x2 Fourier multiplier K^(k) of Eq. (e:project-body-force), as arrays
    (K11, K12, K22) (K21 = K12)."""
    K1o, K2o, KK = symbols(n1, n2)
    kk_odd = K1o ** 2 + K2o ** 2
    ones = np.ones((n1, n2))
    zeros = np.zeros((n1, n2))
    if beta_w == 0.0:  # gamma = 0: no constraint, K = I
        return ones, zeros, ones
    Ah = reg_symbol(n1, n2, regnorm)
    if np.isinf(beta_w):  # w = 0: M = I, Leray projection
        denom = kk_odd.copy()
    else:
        denom = kk_odd + beta_v * Ah / (beta_w * (1.0 + KK))
    nz = kk_odd > 0.0
    coef = np.zeros((n1, n2))
    coef[nz] = 1.0 / denom[nz]
    return 1.0 - coef * K1o * K1o, -coef * K1o * K2o, 1.0 - coef * K2o * K2o


def apply_K(b, regnorm, beta_v, beta_w):
    """K[b] of Eq. (e:project-body-force) (also L[b~] for the quadratic models,
    Eq. (e:inc-control-eq-elim))."""
    n1, n2 = b.shape[-2:]
    K11, K12, K22 = projection_symbol(n1, n2, regnorm, beta_v, beta_w)
    B1, B2 = fft2(b[0]), fft2(b[1])
    return np.stack([_real(ifft2(K11 * B1 + K12 * B2)), _real(ifft2(K12 * B1 + K22 * B2))])


def apply_precond(r, regnorm, beta_v):
    """(beta_v A)^-1 r with the k = 0 symbol of A replaced by 1 (Appendix E and
    its footnote on modifying the kernel).  For the shear-control model the
    paper uses the inverse vector Laplacian, i.e. the H1 symbol (Appendix E)."""
    n1, n2 = r.shape[-2:]
    Ah = reg_symbol(n1, n2, regnorm).copy()
    Ah[0, 0] = 1.0
    return np.stack([_real(ifft2(fft2(r[c]) / (beta_v * Ah))) for c in range(2)])
