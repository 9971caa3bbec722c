"""The GPU solver iterates H2 problems in preconditioned coordinates y = Q v,
Q^ = (beta_v A'^)^(1/2) with A'(0) = 1 (the spectral preconditioner of App. E.2
is P = Q^2).  These FP64 checks, built on the oracle's own operators, pin the
identities that leave Algorithm 2 unchanged there:

  g_y = Q^-1 g            = Pi0 y + Q^-1 K b          (Pi0 drops k = 0)
  H_y = Q^-1 H Q^-1        = Pi0 + Q^-1 K (J^T J) Q^-1
  CG on H_y (no preconditioner) from y = 0 has iterates y_l = Q v_l, where v_l
  are the iterates of PCG on H with preconditioner P, and the same residual
  norms ||Q r_y|| = ||r_v||.
"""
import math

import numpy as np
import pytest

from oracle import spectral as S
from oracle.fft import fft2, ifft2
from oracle.registration import Registration
from paper_1503_00757_gb300 import synth


def _apply(mult, x):
    return np.stack([np.real(ifft2(mult * fft2(x[c]))) for c in range(2)])


def _setup(gamma):
    n, nt, beta = 16, 4, 1e-2
    mT, mR, vs = synth.blobs_pair(n, 1000)
    P = Registration(mT, mR, nt, regnorm=2, beta_v=beta, beta_w=gamma)
    A = S.reg_symbol(n, n, 2).copy()
    A[0, 0] = 1.0
    Q = np.sqrt(beta * A)
    pi0 = np.ones((n, n))
    pi0[0, 0] = 0.0
    return P, Q, pi0, 0.3 * vs


@pytest.mark.parametrize("gamma", [math.inf, 0.0, 1e-3])
def test_gradient_and_hessian_in_preconditioned_coordinates(gamma):
    P, Q, pi0, v = _setup(gamma)
    y = _apply(Q, v)
    g, _ = P.gradient(v)
    Kb = S.apply_K(P.b, 2, P.beta_v, P.beta_w)
    gy = _apply(pi0, y) + _apply(1.0 / Q, Kb)
    assert np.abs(_apply(1.0 / Q, g) - gy).max() < 1e-10 * np.abs(gy).max()
    s = np.random.default_rng(3).standard_normal(v.shape)
    Hs = P.matvec(_apply(1.0 / Q, s))
    Kbt = S.apply_K(P.bt, 2, P.beta_v, P.beta_w)
    Hys = _apply(pi0, s) + _apply(1.0 / Q, Kbt)
    assert np.abs(_apply(1.0 / Q, Hs) - Hys).max() < 1e-10 * np.abs(Hys).max()


@pytest.mark.parametrize("gamma", [math.inf, 1e-3])
def test_cg_in_y_reproduces_pcg_in_v(gamma):
    P, Q, pi0, v = _setup(gamma)
    g, _ = P.gradient(v)
    eta = 1e-6  # run several iterations
    vt_ref, it_ref, relres_ref, _ = P.pcg(g, eta, 6)
    # CG on H_y without a preconditioner, stop test on the v-space residual norm ||Q r||
    gy = _apply(1.0 / Q, g)
    gnorm = S.norm(g)
    yt = np.zeros_like(gy)
    r = -gy
    s = r.copy()
    rz = S.inner(r, r)
    it = 0
    for _ in range(6):
        Hs = _apply(1.0 / Q, P.matvec(_apply(1.0 / Q, s)))
        it += 1
        kappa = rz / S.inner(s, Hs)
        yt = yt + kappa * s
        r = r - kappa * Hs
        if S.norm(_apply(Q, r)) < eta * gnorm:
            break
        rz_new = S.inner(r, r)
        s = r + (rz_new / rz) * s
        rz = rz_new
    assert it == it_ref
    vt = _apply(1.0 / Q, yt)
    assert np.abs(vt - vt_ref).max() < 1e-8 * np.abs(vt_ref).max()
    assert abs(S.norm(_apply(Q, r)) / gnorm - relres_ref) < 1e-8 * relres_ref
