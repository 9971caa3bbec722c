"""Pins for the oracle's transport solves and deformation gradient (CPU only):
closed-form Heun amplification, exact transposition of forward and adjoint
transport, mass conservation, second-order convergence to exact solutions,
and the exact deformation gradient of a shear flow (Eqs. (e:state-eq-elim),
(e:adj-eq-elim), (e:inc-state-eq-elim), (e:def-grad))."""
import numpy as np
import pytest

from oracle import spectral as S
from oracle import transport as T
from paper_1503_00757_gb300 import synth


def test_constant_image_stays_constant():
    rng = np.random.default_rng(1)
    v = synth.velocity(32, 32, 4, 0.5, rng, grad_fraction=0.5)
    m = T.state_solve(np.full((32, 32), 0.7), v, 6)
    assert np.abs(m - 0.7).max() < 1e-14


@pytest.mark.parametrize("k1,k2", [(1, 2), (3, -1), (0, 5)])
def test_constant_velocity_closed_form(k1, k2):
    """Per Fourier mode d_t m^ = -i (k.v) m^; Heun multiplies it by
    R = 1 - i z - z^2/2 per step with z = h k.v."""
    n, nt = 16, 5
    c = np.array([0.37, -0.81])
    v = np.stack([np.full((n, n), c[0]), np.full((n, n), c[1])])
    X1, X2 = S.grid_coords(n, n)
    m0 = np.cos(k1 * X1 + k2 * X2)
    z = (k1 * c[0] + k2 * c[1]) / nt
    R = (1 - 1j * z - 0.5 * z * z) ** nt
    ref = np.real(R * np.exp(1j * (k1 * X1 + k2 * X2)))
    m = T.state_solve(m0, v, nt)
    assert np.abs(m[-1] - ref).max() < 1e-13


def test_constant_velocity_converges_to_integer_shift():
    n = 32
    X1, X2 = S.grid_coords(n, n)
    m0 = np.exp(np.cos(X1) + 0.5 * np.sin(2 * X2))
    s = (2, -1)
    v = np.stack([np.full((n, n), 2 * np.pi * s[0] / n), np.full((n, n), 2 * np.pi * s[1] / n)])
    exact = np.roll(m0, s, axis=(0, 1))
    errs = [np.abs(T.state_solve(m0, v, nt)[-1] - exact).max() for nt in (8, 16, 32)]
    assert errs[-1] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_shear_flow_converges_at_second_order():
    n = 32
    X1, X2 = S.grid_coords(n, n)
    v = np.stack([np.sin(X2), np.zeros((n, n))])

    def m0f(a, b):
        return np.exp(0.8 * np.cos(a)) * (1 + 0.3 * np.sin(b))

    exact = m0f(X1 - np.sin(X2), X2)
    errs = [np.abs(T.state_solve(m0f(X1, X2), v, nt)[-1] - exact).max() for nt in (16, 32, 64)]
    assert errs[-1] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_adjoint_is_exact_transpose_and_conserves_mass():
    rng = np.random.default_rng(2)
    n1, n2, nt = 16, 32, 6
    v = synth.velocity(n1, n2, 5, 0.6, rng, grad_fraction=0.5)
    m0 = rng.standard_normal((n1, n2))
    lam1 = rng.standard_normal((n1, n2))
    fwd = T.state_solve(m0, v, nt)[-1]
    adj = T.adjoint_solve(lam1, v, nt)[0]
    lhs, rhs = S.inner(fwd, lam1), S.inner(m0, adj)
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)
    assert abs(adj.sum() - lam1.sum()) < 1e-10


def test_incremental_state_is_linearization_of_state():
    """m~ from Eq. (e:inc-state-eq-elim) approximates d m_1/dv [v~]; the
    optimize-then-discretize source placement makes the error O(h_t^2)."""
    rng = np.random.default_rng(4)
    n = 32
    mT, _, _ = synth.blobs_pair(n, 1001)
    v = synth.velocity(n, n, 4, 0.4, rng, grad_fraction=0.5)
    vt = synth.velocity(n, n, 4, 0.3, rng, grad_fraction=0.5)
    errs = []
    for nt in (4, 8, 16):
        m = T.state_solve(mT, v, nt)
        mt = T.inc_state_solve(v, vt, T.grad_history(m), nt)[-1]
        eps = 1e-5
        fd = (T.state_solve(mT, v + eps * vt, nt)[-1] - T.state_solve(mT, v - eps * vt, nt)[-1]) / (2 * eps)
        errs.append(np.abs(mt - fd).max() / np.abs(fd).max())
    assert errs[-1] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_defgrad_constant_velocity_is_identity():
    n = 16
    v = np.stack([np.full((n, n), 0.3), np.full((n, n), -0.2)])
    F1 = T.defgrad_solve(v, 4)
    assert np.abs(F1[0, 0] - 1).max() < 1e-14 and np.abs(F1[1, 1] - 1).max() < 1e-14
    assert np.abs(F1[0, 1]).max() < 1e-14 and np.abs(F1[1, 0]).max() < 1e-14


def test_defgrad_shear_flow_exact():
    """v = (sin x2, 0): F(t) = I + t [[0, cos x2], [0, 0]] solves Eq. (e:def-grad)
    and Heun reproduces it exactly (F linear in t, N^2 = 0); det F1 = 1."""
    n = 32
    X1, X2 = S.grid_coords(n, n)
    v = np.stack([np.sin(X2), np.zeros((n, n))])
    F1 = T.defgrad_solve(v, 3)
    assert np.abs(F1[0, 0] - 1).max() < 1e-13
    assert np.abs(F1[0, 1] - np.cos(X2)).max() < 1e-13
    assert np.abs(F1[1, 0]).max() < 1e-13 and np.abs(F1[1, 1] - 1).max() < 1e-13
    det, D = T.defgrad_measures(F1)
    assert np.abs(det - 1).max() < 1e-13
    assert np.abs(D - np.abs(np.cos(X2))).max() < 1e-13


def test_defgrad_incompressible_det_near_one():
    rng = np.random.default_rng(8)
    n = 32
    v = synth.velocity(n, n, 4, 0.5, rng)
    errs = []
    for nt in (8, 16):
        det, _ = T.defgrad_measures(T.defgrad_solve(v, nt))
        errs.append(np.abs(det - 1).max())
    assert errs[1] < 1e-3
    assert errs[0] / errs[1] > 3.0
