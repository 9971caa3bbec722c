"""Pins for the nonlinear Stokes model with a mass source (App. A.2; CPU only).

Per Fourier mode, along k~ and across it, the reduced gradient of App. A.2 is the true
gradient G of J (shear energy + (beta_w/2) <(-Lap + I) w, w> with w = div v + data term)
projected by K~ = I - k~ k~^T / (|k~|^2 m), m = 1 + 2 beta_v eta_bar / (beta_w (1 + |k|^2)):
g~ = K~ G, for any exponent nu.  The paper's Hessian is K~ H_true in the same way.  Hence
<g~, d> = dJ[K~ d] (finite differences of J) and, at a zero-residual point where the
Gauss-Newton Hessian is the Hessian of J, <H v~, d> = d^2 J[v~, K~ d] (mixed differences of J).
Both pin eta_bar in M, the factor 2 beta_v, the eta^ term and the objective's w term; the
first converges with order 2 in h_t.  As beta_w -> inf the reduced gradient tends to the
incompressible one on divergence-free fields."""
import math

import numpy as np
import pytest

from oracle import shear as SH
from oracle import spectral as S
from oracle import transport as T
from oracle.registration import Registration
from paper_1503_00757_gb300 import synth


def _setup(nt, s, bw, seed=1000):
    mT, mR, vs = synth.blobs_pair(32, seed, vmax=0.4, kmax=3)
    P = Registration(mT, mR, nt, regnorm=1, beta_v=1e-2, beta_w=bw, shear=s)
    v = 0.5 * vs + synth.velocity(32, 32, 3, 0.15, np.random.default_rng(5), grad_fraction=1.0)
    return P, v


@pytest.mark.parametrize("s", [-0.5, 0.5])
def test_reduced_gradient_is_projected_true_gradient(s):
    nu = SH.nu_from_shear(s)
    errs = []
    for nt in (4, 8, 16):
        P, v = _setup(nt, s, 1e-2)
        dp = synth.velocity(32, 32, 4, 0.3, np.random.default_rng(7), grad_fraction=0.5)
        d = SH.mass_k(dp, SH.mean_viscosity(v, nu), 1e-2, 1e-2)
        g, _ = P.gradient(v)
        eps = 1e-5
        fd = (P.objective(v + eps * d)[0] - P.objective(v - eps * d)[0]) / (2 * eps)
        errs.append(abs(S.inner(g, dp) - fd) / abs(fd))
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_projection_differs_from_the_incompressible_one():
    """The pin above would pass with a wrong M if the directions were divergence-free; the
    directions here have a gradient part, and the mass-source K~ differs from the Leray
    projection on them by O(1)."""
    v = synth.velocity(32, 32, 4, 0.3, np.random.default_rng(8), grad_fraction=1.0)
    k = SH.mass_k(v, 1.3, 1e-2, 1e-2)
    assert np.linalg.norm(k - SH.leray(v)) > 0.1 * np.linalg.norm(v)


@pytest.mark.parametrize("s", [-0.5, 0.5])
def test_hessian_is_projected_hessian_of_J_at_zero_residual(s):
    nu = SH.nu_from_shear(s)
    mT, _, vs = synth.blobs_pair(32, 1001, vmax=0.4, kmax=3)
    v = 0.5 * vs + synth.velocity(32, 32, 3, 0.15, np.random.default_rng(6), grad_fraction=1.0)
    nt = 16
    mR = T.state_solve(mT, v, nt)[-1]  # zero residual: Gauss-Newton = Hessian of J
    P = Registration(mT, mR, nt, regnorm=1, beta_v=1e-2, beta_w=1e-2, shear=s)
    vt = synth.velocity(32, 32, 4, 0.3, np.random.default_rng(9), grad_fraction=0.5)
    dp = synth.velocity(32, 32, 4, 0.3, np.random.default_rng(10), grad_fraction=0.5)
    d = SH.mass_k(dp, SH.mean_viscosity(v, nu), 1e-2, 1e-2)
    P.gradient(v)
    H = P.matvec(vt)
    e = 1e-3
    J = lambda a, b: P.objective(v + a * vt + b * d)[0]
    mixed = (J(e, e) - J(e, -e) - J(-e, e) + J(-e, -e)) / (4 * e * e)
    assert abs(S.inner(H, dp) - mixed) / abs(mixed) < 5e-3


def test_infinite_beta_w_limit():
    """beta_w -> inf: M -> I and g~ tends to the incompressible reduced gradient (for a
    divergence-free v the two formulations agree, reading in the module docstring)."""
    mT, mR, vs = synth.blobs_pair(32, 1000, vmax=0.4, kmax=3)
    v = 0.5 * vs
    gi, _ = Registration(mT, mR, 8, regnorm=1, beta_v=1e-2, beta_w=math.inf, shear=0.5).gradient(v)
    gm, _ = Registration(mT, mR, 8, regnorm=1, beta_v=1e-2, beta_w=1e12, shear=0.5).gradient(v)
    assert np.linalg.norm(gm - gi) < 1e-8 * np.linalg.norm(gi)


def test_mass_source_shear_solve_converges():
    mT, mR, _ = synth.blobs_pair(32, 1000)
    P = Registration(mT, mR, 8, regnorm=1, beta_v=1e-2, beta_w=1e-2, shear=0.5)
    v, st = P.solve(tol=1e-2)
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2 and st["J"] < st["J0"]
    assert np.abs(S.div(v)).max() > 1e-6  # a mass source: v is not divergence-free
