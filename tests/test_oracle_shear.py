"""Pins for the nonlinear Stokes (shear control) operators of the oracle
(Eqs. (e:shear-control-reg-v), (e:1st-var-reg-v-nls), (e:2nd-var-reg-v-nls)).
References: the linear H1 operator at nu = 1, the closed-form strain and
viscosity of a single shear mode, finite differences of the energy and of
the first variation, and exact symmetry of the second variation."""
import numpy as np
import pytest

from oracle import shear as SH
from oracle import spectral as S
from oracle.registration import Registration
from paper_1503_00757_gb300 import synth


def test_nu_mapping():
    assert SH.nu_from_shear(0.0) == 1.0
    assert SH.nu_from_shear(0.5) == 3.0
    assert abs(SH.nu_from_shear(-0.5) - 1.0 / 3.0) < 1e-15


def test_nu_one_reduces_to_linear_stokes():
    """nu = 1: eta = 1 and Q = 0, so A = -div 2E = -Lap on divergence-free
    band-limited fields (Sec. 2: linear Stokes regularization)."""
    v = synth.velocity(32, 32, 6, 0.5, np.random.default_rng(0))
    Av = SH.first_variation(v, 1.0)
    assert np.abs(Av - S.apply_A(v, S.H1)).max() < 1e-10 * np.abs(Av).max()
    vt = synth.velocity(32, 32, 6, 0.5, np.random.default_rng(1))
    assert np.abs(SH.second_variation(v, vt, 1.0) - S.apply_A(vt, S.H1)).max() < 1e-10 * np.abs(Av).max()


@pytest.mark.parametrize("nu", [1.0 / 3.0, 3.0])
def test_single_mode_strain_and_viscosity(nu):
    n, k = 32, 3
    X1, X2 = S.grid_coords(n, n)
    v = np.stack([np.sin(k * X2), np.zeros((n, n))])
    E11, E12, E22 = SH.strain(v)
    assert np.abs(E11).max() < 1e-12 and np.abs(E22).max() < 1e-12
    assert np.abs(E12 - 0.5 * k * np.cos(k * X2)).max() < 1e-12
    eta = SH.viscosity(v, nu)
    ref = (0.5 * k * k * np.cos(k * X2) ** 2 + SH.EPS ** 2) ** ((1 - nu) / (2 * nu))
    assert np.abs(eta - ref).max() < 1e-10 * ref.max()


@pytest.mark.parametrize("nu", [1.0 / 3.0, 3.0])
def test_first_variation_is_derivative_of_energy(nu):
    rng = np.random.default_rng(2)
    v = synth.velocity(32, 32, 5, 0.4, rng, grad_fraction=0.5)
    d = synth.velocity(32, 32, 5, 0.4, rng, grad_fraction=0.5)
    beta = 1e-3
    eps = 1e-6
    fd = (SH.energy(v + eps * d, nu, beta) - SH.energy(v - eps * d, nu, beta)) / (2 * eps)
    an = beta * S.inner(SH.first_variation(v, nu), d)
    assert abs(fd - an) < 1e-6 * abs(an)


@pytest.mark.parametrize("nu", [1.0 / 3.0, 3.0])
def test_second_variation_is_derivative_of_first_and_symmetric(nu):
    rng = np.random.default_rng(3)
    v = synth.velocity(32, 32, 5, 0.4, rng, grad_fraction=0.5)
    u = synth.velocity(32, 32, 5, 0.4, rng, grad_fraction=0.5)
    w = synth.velocity(32, 32, 5, 0.4, rng, grad_fraction=0.5)
    eps = 1e-6
    fd = (SH.first_variation(v + eps * u, nu) - SH.first_variation(v - eps * u, nu)) / (2 * eps)
    Bu = SH.second_variation(v, u, nu)
    assert np.abs(fd - Bu).max() < 1e-6 * np.abs(Bu).max()
    a, b = S.inner(Bu, w), S.inner(u, SH.second_variation(v, w, nu))
    assert abs(a - b) < 1e-11 * abs(a)
    assert S.inner(Bu, u) > 0


def test_shear_gradient_matches_fd_and_solve_converges():
    mT, mR, vs = synth.blobs_pair(32, 1006, vmax=0.4, kmax=3)
    P = Registration(mT, mR, 16, regnorm=S.H1, beta_v=1e-3, beta_w=np.inf, shear=0.5)
    v = 0.5 * vs
    d = synth.velocity(32, 32, 5, 0.2, np.random.default_rng(4))
    g, _ = P.gradient(v)
    assert np.abs(S.div(g)).max() < 1e-10
    eps = 1e-5
    fd = (P.objective(v + eps * d)[0] - P.objective(v - eps * d)[0]) / (2 * eps)
    assert abs(S.inner(g, d) - fd) < 2e-3 * abs(fd)
    P2 = Registration(mT, mR, 8, regnorm=S.H1, beta_v=1e-2, beta_w=np.inf, shear=0.5)
    v, st = P2.solve(tol=1e-2)
    assert st["status"] == 0 and st["gnorm_rel"] <= 1e-2
    assert np.abs(S.div(v)).max() < 1e-11


def test_shear_requires_h1():
    """The shear model is defined for the H1-type strain energy only; any beta_w is allowed
    (the mass-source variant, App. A.2, is pinned in test_oracle_shear_mass)."""
    with pytest.raises(ValueError):
        Registration(np.zeros((8, 8)), np.zeros((8, 8)), 2, regnorm=S.H2, beta_w=np.inf, shear=0.5)
    Registration(np.zeros((8, 8)), np.zeros((8, 8)), 2, regnorm=S.H1, beta_w=1e-3, shear=0.5)
