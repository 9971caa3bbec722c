"""Pins for the oracle's outer iteration (Algorithm 1): the Armijo backtracking line search,
the steepest-descent fallback, the relative stopping test, the forcing term handed to the
inner solver and the failure statuses.

The registration operators are replaced by a quadratic J(v) = 1/2 <D (v - v*), v - v*> with a
positive diagonal D, whose minimiser, gradient D (v - v*) and Newton step v* - v are known.
The inner solver is replaced by a fake that returns s times the Newton step. Each outcome then
follows in closed form from the Armijo rule J(v + a v~) <= J(v) + c1 a <g, v~>, with a
backtracked from 1 by halving:
* s = 1 (exact step): accepted at a = 1;
* s = 2: a = 1 mirrors v about v* and leaves J unchanged, so it is rejected; a = 1/2 is exact;
* s = 4: rejected at 1 and 1/2, exact at 1/4;
* s = 1/2 (half step): accepted at a = 1, and ||g|| halves every iteration;
* s = -1 (ascent direction): replaced by -P^-1 g, which is exact here;
* c1 > 1: no step can satisfy the rule.

Algorithm 2's PCG runs on a diagonal operator with k distinct eigenvalues. There CG must
terminate after exactly k iterations, since the Krylov space is then exhausted. With the exact
inverse as preconditioner it must terminate after one."""
import math

import numpy as np
import pytest

from oracle import spectral as S
from oracle.registration import STATUS_LINESEARCH, STATUS_MAXIT, STATUS_OK, Registration


class Quadratic(Registration):
    """A Registration whose objective, gradient, inner solve and preconditioner are a
    quadratic with a known minimiser; the outer loop is the oracle's own."""

    def __init__(self, n=16, s=1.0, seed=0):
        rng = np.random.default_rng(seed)
        self.mT = np.zeros((n, n))
        self.mR = np.zeros((n, n))
        self.m = [self.mT]
        self.nt = 4
        self.n_pde = 0
        self.D = 0.5 + rng.random((2, n, n))
        self.vstar = rng.standard_normal((2, n, n))
        self.s = s
        self.etas = []

    def nt_for(self, v, policy, c_max=0.25):
        return self.nt

    def objective(self, v, nt=None):
        e = v - self.vstar
        return 0.5 * S.inner(self.D * e, e), [self.mT]

    def gradient(self, v, nt=None):
        e = v - self.vstar
        return self.D * e, 0.5 * S.inner(self.D * e, e)

    def precond(self, r):
        return r / self.D

    def pcg(self, g, eta, maxit):
        self.etas.append(eta)
        return -self.s * g / self.D, 1, 0.0, False


@pytest.mark.parametrize("s,n_ls", [(1.0, 1), (2.0, 2), (4.0, 3)])
def test_armijo_backtracks_to_the_exact_step(s, n_ls):
    P = Quadratic(s=s)
    v, st = P.solve(tol=1e-2)
    assert st["status"] == STATUS_OK
    assert st["n_newton"] == 1 and st["n_ls"] == n_ls
    assert np.abs(v - P.vstar).max() < 1e-12
    assert st["gnorm_rel"] < 1e-12


def test_ascent_direction_falls_back_to_preconditioned_steepest_descent():
    P = Quadratic(s=-1.0)
    v, st = P.solve(tol=1e-2)
    assert st["status"] == STATUS_OK and st["n_newton"] == 1 and st["n_ls"] == 1
    assert np.abs(v - P.vstar).max() < 1e-12


def test_half_steps_stop_at_the_relative_tolerance_with_the_forcing_sequence():
    # ||g_k|| / ||g_0|| = 2^-k; the test ||g_k|| / ||g_ref|| <= 1e-2 first holds at k = 7
    P = Quadratic(s=0.5)
    v, st = P.solve(tol=1e-2)
    assert st["status"] == STATUS_OK and st["n_newton"] == 7 and st["n_ls"] == 7
    assert np.abs(v - (1 - 2.0 ** -7) * P.vstar).max() < 1e-12
    assert abs(st["gnorm_rel"] - 2.0 ** -7) < 1e-12
    # the forcing term of Algorithm 2 at iteration k, min(0.5, sqrt(||g_k|| / ||g_0||))
    assert np.allclose(P.etas, [min(0.5, math.sqrt(2.0 ** -k)) for k in range(7)], rtol=0, atol=1e-12)
    assert P.etas[0] == 0.5 and P.etas[3] < 0.5


def test_line_search_failure_and_newton_cap():
    P = Quadratic(s=1.0)
    v, st = P.solve(tol=1e-2, c1=1.5, max_ls=12)
    assert st["status"] == STATUS_LINESEARCH and st["n_ls"] == 12 and st["n_newton"] == 0
    assert not v.any()  # no step taken from v = 0
    P = Quadratic(s=0.5)
    v, st = P.solve(tol=1e-2, maxit_newton=3)
    assert st["status"] == STATUS_MAXIT and st["n_newton"] == 3
    assert np.abs(v - 0.875 * P.vstar).max() < 1e-12


def test_warm_start_keeps_the_zero_start_reference():
    # from v0 = v*/2 the gradient is half of g(0); half steps reach 1e-2 of ||g(0)|| in 6 steps
    P = Quadratic(s=0.5)
    v, st = P.solve(v0=0.5 * P.vstar, tol=1e-2)
    assert st["status"] == STATUS_OK and st["n_newton"] == 6
    assert abs(st["gnorm_rel"] - 2.0 ** -7) < 1e-12
    # the forcing term is relative to the gradient at the warm start
    assert P.etas[0] == 0.5 and abs(P.etas[2] - 0.5) < 1e-12 and abs(P.etas[3] - math.sqrt(0.125)) < 1e-12


class Diagonal(Registration):
    """A Registration whose Hessian is a diagonal operator with a chosen set of eigenvalues
    and whose preconditioner is chosen per test; Algorithm 2's loop is the oracle's own."""

    def __init__(self, eigs, n=16, precond_exact=False, seed=1):
        rng = np.random.default_rng(seed)
        self.lam = rng.choice(np.asarray(eigs, dtype=np.float64), size=(2, n, n))
        self.lam.flat[: len(eigs)] = eigs  # every eigenvalue present
        self.exact = precond_exact
        self.n_pde = 0

    def matvec(self, vt):
        return self.lam * vt

    def precond(self, r):
        return r / self.lam if self.exact else r


@pytest.mark.parametrize("eigs", [[2.0], [1.0, 3.0], [0.5, 2.0, 7.0], [1.0, 2.0, 4.0, 8.0, 16.0]])
def test_pcg_terminates_after_as_many_iterations_as_distinct_eigenvalues(eigs):
    # the Krylov space of a matrix with k distinct eigenvalues is exhausted after k steps
    P = Diagonal(eigs)
    g = np.random.default_rng(2).standard_normal(P.lam.shape)
    vt, it, relres, hit = P.pcg(g, 1e-10, 50)
    assert it == len(eigs) and not hit and relres < 1e-10
    assert np.abs(vt + g / P.lam).max() < 1e-9 * np.abs(g / P.lam).max()


def test_pcg_with_the_exact_preconditioner_takes_one_iteration_and_caps():
    P = Diagonal([0.5, 2.0, 7.0, 11.0], precond_exact=True)
    g = np.random.default_rng(3).standard_normal(P.lam.shape)
    vt, it, relres, hit = P.pcg(g, 1e-10, 50)
    assert it == 1 and not hit and np.abs(vt + g / P.lam).max() < 1e-12
    P = Diagonal([0.5, 2.0, 7.0, 11.0])
    vt, it, relres, hit = P.pcg(g, 1e-10, 2)
    assert it == 2 and hit and relres > 1e-6
