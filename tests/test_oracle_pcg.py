"""Pins of the oracle's fixed-count Jacobi-PCG (the CPU baseline's and the
reference arm's timed loop) against properties that fix its iterates.

The paper names no linear solver (it reports residual levels only,
Sec. 4.1.1); the oracle runs textbook Jacobi-preconditioned conjugate
gradients on the pinned GFM system of Sec. 3.1.  The k-th PCG iterate from
x0 = 0 is characterised without reference to the recurrence: it is the
Galerkin (A-norm optimal) approximation of A^-1 b from the preconditioned
Krylov space K_k(M^-1 A, M^-1 b), M = diag(A).  The tests build that space
with Arnoldi and solve the small projected system directly, check the
returned residual norm against ||b - A x_k|| formed densely, check finite
termination on a tiny system against a dense solve, and plant the two
mistakes a fixed-count loop is most likely to carry (Jacobi weights dropped,
r.z never updated) to show that the pin catches them.
"""
import numpy as np
import pytest

import cases
import oracle


def _gfm_system(nx=12, ny=8, seed=21):
    """A small two-phase tank: density ratio 1000 across an interface row."""
    c = cases.box_case(nx, ny, 1, seed=seed, ka=0.12)
    fc = oracle.faces(c)
    sy = oracle.assemble(c, fc)
    return c, sy


def _krylov_galerkin(A, b, k):
    """A-norm optimal x in K_k(M^-1 A, M^-1 b), M = diag(A): an orthonormal
    basis by Arnoldi (modified Gram-Schmidt, twice), then the k x k
    projected system V^T A V y = V^T b."""
    dinv = 1.0 / np.diag(A)
    n = b.size
    V = np.zeros((n, k))
    v = dinv * b
    for j in range(k):
        for _ in range(2):
            for i in range(j):
                v = v - (V[:, i] @ v) * V[:, i]
        V[:, j] = v / np.linalg.norm(v)
        v = dinv * (A @ V[:, j])
    y = np.linalg.solve(V.T @ A @ V, V.T @ b)
    return V @ y


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_pcg_fixed_iterate_is_the_krylov_galerkin_solution(k):
    _, sy = _gfm_system()
    A = sy.dense()
    x_k, _ = oracle.pcg_fixed(sy, k)
    x_ref = _krylov_galerkin(A, sy.b, k)
    err = np.linalg.norm(x_k - x_ref) / np.linalg.norm(x_ref)
    assert err <= 1e-8, (k, err)


def test_pcg_fixed_returns_the_residual_norm_of_its_iterate():
    _, sy = _gfm_system()
    A = sy.dense()
    for k in (1, 4, 10, 25):
        x_k, rr = oracle.pcg_fixed(sy, k)
        true = np.linalg.norm(sy.b - A @ x_k)
        assert abs(rr - true) <= 1e-9 * np.linalg.norm(sy.b), (k, rr, true)


def test_pcg_fixed_reaches_the_dense_solution_in_n_steps():
    """Finite termination: on a well-conditioned tiny system (single phase,
    so the density ratio does not stretch the spectrum) n iterations give
    the direct solution up to rounding."""
    c = cases.box_case(4, 3, 1, seed=3, ka=0.0)
    alpha = np.ones(c.n)
    sy = oracle.assemble(c, oracle.faces(c, alpha=alpha))
    x_direct = np.linalg.solve(sy.dense(), sy.b)
    x_n, rr = oracle.pcg_fixed(sy, c.n)
    assert np.linalg.norm(x_n - x_direct) <= 1e-10 * np.linalg.norm(x_direct)
    assert rr <= 1e-10 * np.linalg.norm(sy.b)


def test_pcg_fixed_from_a_start_vector():
    """From x0 the iterate is x0 plus the Galerkin correction of r0 = b - A x0."""
    _, sy = _gfm_system(seed=5)
    A = sy.dense()
    x0 = np.random.default_rng(0).standard_normal(sy.n)
    x_k, _ = oracle.pcg_fixed(sy, 4, x0=x0)
    x_ref = x0 + _krylov_galerkin(A, sy.b - A @ x0, 4)
    assert np.linalg.norm(x_k - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_pcg_fixed_agrees_with_the_converging_oracle_solve():
    """Run long enough, the fixed-count loop lands where the stopping PCG
    (checked against dense Cholesky elsewhere) lands."""
    c = cases.make_case(1)
    sy = oracle.assemble(c, oracle.faces(c))
    x_conv, it, rel, st = oracle.pcg(sy, rtol=1e-12)
    assert st == 0
    x_k, rr = oracle.pcg_fixed(sy, it)
    assert np.linalg.norm(x_k - x_conv) <= 1e-9 * np.linalg.norm(x_conv)


@pytest.mark.parametrize("mut", [oracle.MUT_PCG_NO_PRECOND, oracle.MUT_PCG_STALE_RZ])
def test_planted_pcg_mistakes_fail_the_galerkin_pin(mut):
    _, sy = _gfm_system()
    A = sy.dense()
    worst = 0.0
    for k in (2, 3, 5):
        x_bad, _ = oracle.pcg_fixed(sy, k, mutate=mut)
        x_ref = _krylov_galerkin(A, sy.b, k)
        worst = max(worst, np.linalg.norm(x_bad - x_ref) / np.linalg.norm(x_ref))
    assert worst > 1e-4, worst
