"""Three-dimensional gradient and Gauss-Newton matvec on the GPU (reg3_*) against the FP64
oracle (oracle/reg3d.py) on the same seeded inputs, element by element in relative L2.

Tolerance: the FP32 transforms (radix-2, rounding ~ u log2(n) per transform) and nt Heun
steps keep each operator application within 1e-5 of FP64 on coarse axes; every spectral
derivative multiplies the transforms' rounding by up to k_max = n / 2, and the sums
g = beta_v A v + K b and H v~ = beta_v A v~ + K b~ lose the conditioning
c = (||beta_v A x|| + ||b||) / ||y|| of the cancellation between their terms.  So the sums are
held to max(1, c) (2e-5 + 2 u (n / 2) log2(n)), n the longest axis, u = 2^-24 (the factor 2:
the matvec differentiates twice along its chain, grad m in the source and div in the
adjoint).  On 16-point axes the rounding term is 2e-6; on a 256-point axis 1.2e-4.  J: 2e-5.
Shapes cover cubes, anisotropic boxes and 256-point axes (the largest shared-memory FFT tile)
along each axis."""
import math

import numpy as np
import pytest

from oracle import reg3d as R

from .gpu_util import check, to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _smooth(shape, rng, kmax, amp):
    """Random real trigonometric field with modes |k_i| <= kmax, scaled to max |f| = amp."""
    X = R.grid_coords(shape)
    f = np.zeros(shape)
    for _ in range(12):
        k = rng.integers(-kmax, kmax + 1, size=3)
        f += rng.standard_normal() * np.cos(sum(kc * Xc for kc, Xc in zip(k, X)) + rng.uniform(0, 2 * np.pi))
    return amp * f / np.abs(f).max()


def _inputs(shape, seed, nt):
    """Images, a velocity within the explicit scheme's stability (CFL number max|v| h_t k_max
    <= 1/2, k_max = max(n) / 2: Heun amplifies modes beyond |z| = 2 and the FP32 and FP64
    runs would diverge in amplified rounding) and a direction."""
    rng = np.random.default_rng(seed)
    X1, X2, X3 = R.grid_coords(shape)
    bump = lambda c: np.exp(-4.0 * sum(np.sin((Xi - ci) / 2) ** 2 for Xi, ci in zip((X1, X2, X3), c)))
    mT = bump((3.0, 3.1, 2.9)) + 0.5 * bump((2.0, 4.0, 3.5))
    mR = bump((3.25, 2.9, 3.2)) + 0.5 * bump((2.2, 3.8, 3.3))
    vmax = min(0.3, 0.5 * nt / (max(shape) / 2))
    v = np.stack([_smooth(shape, rng, 2, vmax) for _ in range(3)])
    vt = np.stack([_smooth(shape, rng, 3, 0.2) for _ in range(3)])
    return mT, mR, v, vt


CASES = [
    ((16, 16, 16), 4, math.inf),
    ((16, 8, 32), 4, 0.0),
    ((32, 16, 8), 3, 1e-3),
    ((8, 8, 256), 2, math.inf),
    ((256, 8, 8), 2, 1e-3),
    ((8, 256, 16), 2, 0.0),
]


@pytest.mark.parametrize("shape,nt,beta_w", CASES)
def test_gradient_and_matvec_match_oracle(shape, nt, beta_w):
    import torch
    from paper_1503_00757_gb300.binding import Context3D
    beta = 1e-2
    mT, mR, v, vt = _inputs(shape, 7000 + sum(shape) + nt, nt)
    P = R.Registration3D(mT, mR, nt, beta, beta_w)
    g_ref, J_ref = P.gradient(v)
    H_ref = P.matvec(vt)
    ctx = Context3D(*shape, nt, beta=beta, gamma=beta_w)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    g = torch.empty(3, *shape, device="cuda")
    J = ctx.gradient(to_gpu(v), g)
    H = torch.empty(3, *shape, device="cuda")
    ctx.hessian_matvec(to_gpu(vt), H)
    torch.cuda.synchronize()
    ctx.close()
    tag = f"{shape} nt={nt} beta_w={beta_w}"
    n = max(shape)
    base = 2e-5 + 2.0 * 2.0 ** -24 * (n / 2) * math.log2(n)
    check(f"3-D J ({tag})", abs(J - J_ref) / abs(J_ref), 2e-5)
    c_g = (R.norm(beta * R.apply_A(v)) + R.norm(P.b)) / R.norm(g_ref)
    e_g = np.linalg.norm(to_np(g) - g_ref) / np.linalg.norm(g_ref)
    check(f"3-D gradient ({tag})", e_g, base * max(1.0, c_g), cond=c_g)
    c_h = (R.norm(beta * R.apply_A(vt)) + R.norm(P.bt)) / R.norm(H_ref)
    e_h = np.linalg.norm(to_np(H) - H_ref) / np.linalg.norm(H_ref)
    check(f"3-D Gauss-Newton matvec ({tag})", e_h, base * max(1.0, c_h), cond=c_h)


def test_matvec_needs_a_gradient_first():
    import torch
    from paper_1503_00757_gb300.binding import Context3D
    ctx = Context3D(8, 8, 8, 2)
    x = torch.zeros(3, 8, 8, 8, device="cuda")
    with pytest.raises(Exception):
        ctx.hessian_matvec(x, x.clone())
    with pytest.raises(Exception):
        ctx.gradient(x, x.clone())  # no images yet
    ctx.close()


@pytest.mark.parametrize("beta_w", [math.inf, 0.0])
def test_solve_matches_oracle_solve(beta_w):
    """Algorithm 1 on the GPU against the oracle's Algorithm 1 (16^3, nt = 4, tol 1e-2): the
    same Newton count, the stopping test confirmed by the oracle's gradient at the GPU's v
    (<= 1.1e-2 ||g(0)||: 10 % slack for the FP32 gradient the GPU stopped on), and v within
    the spread two solves that both pass the test may have (compared at 2e-2: inexact PCG
    solves determine v only to kappa(H) times the tolerance)."""
    import torch
    from paper_1503_00757_gb300.binding import Context3D
    shape, nt, beta = (16, 16, 16), 4, 1e-2
    mT, mR, _, _ = _inputs(shape, 7100, nt)
    P = R.Registration3D(mT, mR, nt, beta, beta_w)
    v_ref, st_ref = R.solve(P, tol=1e-2)
    assert st_ref["status"] == 0
    ctx = Context3D(*shape, nt, beta=beta, gamma=beta_w)
    ctx.set_images(to_gpu(mT), to_gpu(mR))
    v = torch.empty(3, *shape, device="cuda")
    st = ctx.solve(v, tol=1e-2)
    ctx.close()
    assert st["rc"] == 0 and st["status"] == 0 and st["gnorm_rel"] <= 1e-2
    assert st["n_newton"] == st_ref["n_newton"]
    vg = to_np(v)
    g0 = R.norm(P.gradient(np.zeros_like(v_ref))[0])
    check(f"3-D solve: oracle ||g(v)|| / ||g(0)|| at the GPU's v (beta_w={beta_w})", R.norm(P.gradient(vg)[0]) / g0,
          1.1e-2)
    check(f"3-D solve: v against the oracle's solve (beta_w={beta_w})",
          np.linalg.norm(vg - v_ref) / np.linalg.norm(v_ref), 2e-2)


def test_contexts_of_different_sizes_coexist():
    """A large-tile context stays usable after a smaller one is created (the FFT pass's
    shared-memory opt-in is shared by all contexts of the process)."""
    import torch
    from paper_1503_00757_gb300.binding import Context3D
    shape, nt = (8, 8, 256), 2
    mT, mR, v, _ = _inputs(shape, 7200, nt)
    big = Context3D(*shape, nt, beta=1e-2)
    small = Context3D(16, 16, 16, 2, beta=1e-2)
    big.set_images(to_gpu(mT), to_gpu(mR))
    g = torch.empty(3, *shape, device="cuda")
    J = big.gradient(to_gpu(v), g)
    torch.cuda.synchronize()
    small.close()
    big.close()
    g_ref, J_ref = R.Registration3D(mT, mR, nt, 1e-2).gradient(v)
    assert abs(J - J_ref) < 2e-5 * abs(J_ref)
    assert np.linalg.norm(to_np(g) - g_ref) < 2e-4 * np.linalg.norm(g_ref)
