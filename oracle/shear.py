"""Nonlinear Stokes ("shear control") regularization (oracle; test
infrastructure only).

Model (Sec. 2, Eq. (e:shear-control-reg-v)): with the strain rate tensor
E[v] = (grad v + grad v^T)/2 and flow-law exponent nu > 0,

    R[v] = beta_v * (2 nu / (nu + 1)) * int (E:E + eps^2)^((1 + nu) / (2 nu)) dx.

Readings the paper leaves open:
  * Normalization: the objective carries beta_v times the printed seminorm
    expression (not beta_v / 2), so that its first variation is exactly
    beta_v A[v] with A[v] = -div(2 eta E[v]) of Eq. (e:1st-var-reg-v-nls) and
    at nu = 1 it reduces to (beta_v / 2)|v|^2_H1 for divergence-free v.
  * The viscosity eta = (E:E)^((1 - nu) / (2 nu)) is singular (nu > 1) or
    degenerate (nu < 1) at E = 0, e.g. at the initial guess v = 0
    (Algorithm 1).  Both sides use eta = (E:E + eps^2)^((1 - nu) / (2 nu)) with
    eps = 1e-3, which keeps R, A and B consistent derivatives of each other.
  * Mapping of the configuration knob s in (-1, 1) to the exponent:
    nu = (1 + s) / (1 - s) (s = 0: linear Stokes, s = 1/2: nu = 3, the paper's
    shear-thinning value, s = -1/2: nu = 1/3, shear thickening).
  * Incompressible case (w = 0): for divergence-free v and v~ the paper's
    K[b, v] and L(v)[b~, v~] (Eqs. (e:control-eq-ns),
    (e:project-inc-body-force-nls)) equal the Leray projection of
    beta_v A[v] + b and beta_v B(v)[v~] + b~: the mean-viscosity parts cancel
    because div div E[u] = Lap div u = 0.
  * Mass source (0 < beta_w < inf; App. A.2, no results in the paper):
    eta = eta^ + eta_bar with eta_bar the mean of eta over the domain;
    g~ = -div(2 beta_v eta E[v]) + grad M^-1 Lap^-1 div(div(2 beta_v eta^ E[v]) - b) + b,
    M = 2 beta_v eta_bar (beta_w(-Lap + I))^-1 + I; the Hessian applies
    beta_v B(v)[v~] + grad M^-1 Lap^-1 div(div(2 beta_v (eta^ + eta Q) E[v~]) - b~) + b~
    with the M of the linearization point (Eq. (e:project-inc-body-force-nls)).
    In Fourier, grad M^-1 Lap^-1 div x = P x with P = k~ k~^T / (|k~|^2 m),
    m = 1 + 2 beta_v eta_bar / (beta_w (1 + |k|^2)) (odd symbol k~ for grad and
    div, even |k|^2 in the H1 norm of w, as for the quadratic models); P = 0
    where k~ = 0.

Second variation, Eq. (e:2nd-var-reg-v-nls):
    B(v)[v~] = -div 2 eta (I + Q) E[v~],  Q = ((1 - nu)/nu) E (x) E / (E:E + eps^2).
"""
import numpy as np

from .fft import fft2, ifft2
from .spectral import grad, apply_K, spacing, symbols, H1

EPS = 1.0e-3


def nu_from_shear(s):
    return (1.0 + s) / (1.0 - s)


def strain(v):
    """(E11, E12, E22) of E[v] = (grad v + grad v^T) / 2."""
    g0 = grad(v[0])  # (d1 v1, d2 v1)
    g1 = grad(v[1])  # (d1 v2, d2 v2)
    return g0[0], 0.5 * (g0[1] + g1[0]), g1[1]


def contract(E, F):
    """E : F for symmetric 2x2 tensors given as (11, 12, 22)."""
    return E[0] * F[0] + 2.0 * E[1] * F[1] + E[2] * F[2]


def viscosity(v, nu):
    E = strain(v)
    return (contract(E, E) + EPS ** 2) ** ((1.0 - nu) / (2.0 * nu))


def div_tensor(T):
    """(div T)_a = sum_c d_c T_ac for a symmetric tensor T = (T11, T12, T22)."""
    gT11, gT12, gT22 = grad(T[0]), grad(T[1]), grad(T[2])
    return np.stack([gT11[0] + gT12[1], gT12[0] + gT22[1]])


def energy(v, nu, beta_v):
    E = strain(v)
    p = (1.0 + nu) / (2.0 * nu)
    h1, h2 = spacing(v.shape)
    return beta_v * (2.0 * nu / (nu + 1.0)) * h1 * h2 * float(np.sum((contract(E, E) + EPS ** 2) ** p))


def first_variation(v, nu):
    """A[v] = -div(2 eta[v] E[v]), Eq. (e:1st-var-reg-v-nls)."""
    E = strain(v)
    eta = (contract(E, E) + EPS ** 2) ** ((1.0 - nu) / (2.0 * nu))
    return -div_tensor(tuple(2.0 * eta * e for e in E))


def second_variation(v, vt, nu):
    """B(v)[v~] = -div 2 eta (I + Q) E[v~], Eq. (e:2nd-var-reg-v-nls)."""
    E = strain(v)
    Et = strain(vt)
    ee = contract(E, E) + EPS ** 2
    eta = ee ** ((1.0 - nu) / (2.0 * nu))
    q = ((1.0 - nu) / nu) * contract(E, Et) / ee
    T = tuple(2.0 * eta * (et + q * e) for e, et in zip(E, Et))
    return -div_tensor(T)


def leray(b):
    return apply_K(b, H1, 1.0, np.inf)


def mean_viscosity(v, nu):
    """eta_bar[v] = (1 / #Omega) int eta[v] dx (the discrete mean over the nodes)."""
    return float(np.mean(viscosity(v, nu)))


def mass_p(x, eta_bar, beta_v, beta_w):
    """P x = grad M^-1 Lap^-1 div x of the mass-source elimination (App. A.2), a 2x2 Fourier
    multiplier k~ k~^T / (|k~|^2 m), m = 1 + 2 beta_v eta_bar / (beta_w (1 + |k|^2))."""
    n1, n2 = x.shape[-2:]
    K1o, K2o, KK = symbols(n1, n2)
    kko = K1o ** 2 + K2o ** 2
    m = 1.0 + 2.0 * beta_v * eta_bar / (beta_w * (1.0 + KK))
    c = np.zeros((n1, n2))
    nz = kko > 0.0
    c[nz] = 1.0 / (kko[nz] * m[nz])
    X1, X2 = fft2(x[0]), fft2(x[1])
    proj = c * (K1o * X1 + K2o * X2)
    return np.stack([np.real(ifft2(K1o * proj)), np.real(ifft2(K2o * proj))])


def mass_k(x, eta_bar, beta_v, beta_w):
    """K~ x = x - P x: the projection that maps the true gradient of J onto the reduced
    gradient (and the true Hessian onto the paper's Hessian) of the mass-source model."""
    return x - mass_p(x, eta_bar, beta_v, beta_w)


def reduced_gradient_mass(v, b, nu, beta_v, beta_w):
    """g~ of the nonlinear Stokes model with a mass source (App. A.2)."""
    E = strain(v)
    eta = (contract(E, E) + EPS ** 2) ** ((1.0 - nu) / (2.0 * nu))
    eta_bar = float(np.mean(eta))
    A = -div_tensor(tuple(2.0 * beta_v * eta * e for e in E))
    S = div_tensor(tuple(2.0 * beta_v * (eta - eta_bar) * e for e in E))
    return A + mass_p(S - b, eta_bar, beta_v, beta_w) + b


def hessian_mass(v, vt, bt, nu, beta_v, beta_w):
    """beta_v B(v)[v~] + L(v)[b~, v~] of Eq. (e:project-inc-body-force-nls) with the mass
    source: L = P(div(2 beta_v (eta^ + eta Q) E[v~]) - b~) + b~, eta_bar and P at v."""
    E = strain(v)
    Et = strain(vt)
    ee = contract(E, E) + EPS ** 2
    eta = ee ** ((1.0 - nu) / (2.0 * nu))
    eta_bar = float(np.mean(eta))
    q = ((1.0 - nu) / nu) * contract(E, Et) / ee
    Bv = -div_tensor(tuple(2.0 * beta_v * eta * (et + q * e) for e, et in zip(E, Et)))
    S = div_tensor(tuple(2.0 * beta_v * ((eta - eta_bar) * et + eta * q * e) for e, et in zip(E, Et)))
    return Bv + mass_p(S - bt, eta_bar, beta_v, beta_w) + bt
