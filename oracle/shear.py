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
  * Only the incompressible case (w = 0) is supported; the paper reports no
    results for the mass-source variant (Sec. 5.2).  For divergence-free
    v and v~ the paper's K[b, v] and L(v)[b~, v~] (Eqs. (e:control-eq-ns),
    (e:project-inc-body-force-nls)) equal the Leray projection of
    beta_v A[v] + b and beta_v B(v)[v~] + b~: the mean-viscosity parts cancel
    because div div E[u] = Lap div u = 0.

Second variation, Eq. (e:2nd-var-reg-v-nls):
    B(v)[v~] = -div 2 eta (I + Q) E[v~],  Q = ((1 - nu)/nu) E (x) E / (E:E + eps^2).
"""
import numpy as np

from .spectral import grad, apply_K, spacing, H1

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
