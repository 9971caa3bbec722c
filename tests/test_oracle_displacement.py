"""Pins for the oracle's displacement field (Eq. (e:displacement)) and label-overlap measures
(App. F table; Sec. 5 label evaluation), CPU only.

Displacement: a constant velocity and the shear flow v = (sin x2, 0) give u(t) = t v exactly
(grad u . v = 0 along both; Heun is exact for a solution linear in t); second-order
convergence in h_t on a general field; and consistency with the independently pinned
deformation gradient: F_1 = (I - grad u_1)^-1 up to O(h_t^2) (both describe the same map,
F_1 = (grad y)^-1 with y = x - u_1, App. D).

Overlap: two axis-aligned rectangles whose intersection, union and differences are counted by
hand; identical and disjoint maps; a zero velocity leaves the smoothed, thresholded labels of a
large smooth region unchanged."""
import numpy as np

from oracle import measures as M
from oracle import spectral as S
from oracle import transport as T
from paper_1503_00757_gb300 import synth


def test_constant_velocity_displacement_is_exact():
    n = 32
    v = np.stack([np.full((n, n), 0.3), np.full((n, n), -0.2)])
    for nt in (1, 3, 8):
        u = T.displacement_solve(v, nt)
        assert np.abs(u - v).max() < 1e-14


def test_shear_flow_displacement_is_exact():
    n = 32
    X1, X2 = S.grid_coords(n, n)
    v = np.stack([np.sin(X2), np.zeros((n, n))])
    u = T.displacement_solve(v, 4)
    assert np.abs(u - v).max() < 1e-13


def _field(n, seed):
    return synth.velocity(n, n, 3, 0.5, np.random.default_rng(seed), grad_fraction=0.4)


def test_displacement_converges_second_order():
    n = 32
    v = _field(n, 5)
    ref = T.displacement_solve(v, 512)
    errs = [np.abs(T.displacement_solve(v, nt) - ref).max() for nt in (8, 16, 32)]
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_displacement_agrees_with_deformation_gradient():
    n = 32
    v = _field(n, 6)
    errs = []
    for nt in (8, 16, 32):
        u = T.displacement_solve(v, nt)
        gu = np.stack([S.grad(u[0]), S.grad(u[1])])  # gu[a, b] = d_b u_a
        A = np.zeros_like(gu)
        A[0, 0], A[1, 1] = 1.0 - gu[0, 0], 1.0 - gu[1, 1]
        A[0, 1], A[1, 0] = -gu[0, 1], -gu[1, 0]
        det = A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]
        Finv = np.stack([np.stack([A[1, 1], -A[0, 1]]), np.stack([-A[1, 0], A[0, 0]])]) / det
        F1 = T.defgrad_solve(v, nt)
        errs.append(np.abs(F1 - Finv).max())
    assert errs[-1] < 1e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_overlap_of_two_rectangles():
    LT = np.zeros((16, 16), bool)
    LR = np.zeros((16, 16), bool)
    LT[0:8, 0:8] = True    # 64 nodes
    LR[4:12, 0:8] = True   # 64 nodes; 32 shared, 96 in the union
    jsc, dsc, fpe, fne = M.overlap(LT, LR)
    assert (jsc, dsc, fpe, fne) == (32 / 96, 64 / 128, 32 / 64, 32 / 64)
    assert M.overlap(LT, LT) == (1.0, 1.0, 0.0, 0.0)
    far = np.zeros((16, 16), bool)
    far[10:16, 10:16] = True
    assert M.overlap(LT, far) == (0.0, 0.0, 1.0, 1.0)


def test_zero_velocity_keeps_a_stripe():
    """A stripe of rows has straight edges midway between nodes: the Gaussian-smoothed
    indicator is symmetric about 0.5 there, so thresholding returns the stripe, and a zero
    velocity transports nothing.  A shift of the stripe by whole rows under a constant velocity
    (v = 2 pi s / n, nt large) moves the overlap to the hand count."""
    n = 64
    L = np.zeros((n, n))
    L[16:40, :] = 1.0
    assert M.label_overlap(L, L, np.zeros((2, n, n)), 4) == (1.0, 1.0, 0.0, 0.0)
    v = np.stack([np.full((n, n), 2 * np.pi * 4 / n), np.zeros((n, n))])  # 4 rows in t = 1
    jsc, dsc, fpe, fne = M.label_overlap(L, L, v, 64)
    assert (jsc, dsc, fpe, fne) == (20 / 28, 40 / 48, 4 / 24, 4 / 24)


def test_gaussian_smoothing_symbol():
    n = 32
    X1, X2 = S.grid_coords(n, n)
    f = np.cos(3 * X1 + 2 * X2)
    s = 0.2
    assert np.abs(M.gaussian_smooth(f, s) - np.exp(-0.5 * s * s * 13) * f).max() < 1e-13
