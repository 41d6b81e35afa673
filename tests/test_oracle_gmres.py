"""Pins of the oracle's GMRES (Sec. 6: restarted GMRES with modified Gram-Schmidt, right
preconditioning) against properties that fix it independently of its own code: finite
termination, the one-step solve with the exact inverse as preconditioner, and the minimal
residual over the Krylov space computed by brute force (explicit Krylov basis + least squares)."""
import numpy as np
import pytest

from oracle import gmres as gm


def _system(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 4 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def test_finite_termination_without_restart():
    # in exact arithmetic GMRES solves an n x n system in at most n steps
    A, b = _system(12, 1)
    x, its, res = gm.gmres_one(A, b, lambda v: v, rtol=1e-12, restart=12, max_iters=12)
    assert its <= 12 and res <= 1e-10
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-9 * np.linalg.norm(x))


def test_exact_inverse_preconditioner_takes_one_step():
    # A M^-1 = I: the first Krylov vector already spans the solution
    A, b = _system(20, 2)
    Ainv = np.linalg.inv(A)
    x, its, res = gm.gmres_one(A, b, lambda v: Ainv @ v, rtol=1e-10, restart=30, max_iters=30)
    assert its == 1 and res <= 1e-10


@pytest.mark.parametrize("k", [1, 3, 6])
def test_iterate_minimises_the_residual_over_the_krylov_space(k):
    # after k steps (no restart) the iterate minimises ||b - A x|| over x in K_k(A, b); the
    # minimum is computed here from the explicit Krylov basis [b, A b, ..., A^(k-1) b]
    A, b = _system(16, 3 + k)
    x, its, _ = gm.gmres_one(A, b, lambda v: v, rtol=0.0, restart=30, max_iters=k)
    assert its == k
    K = np.empty((16, k), complex)
    v = b.copy()
    for j in range(k):
        K[:, j] = v
        v = A @ v
    c, *_ = np.linalg.lstsq(A @ K, b, rcond=None)
    best = np.linalg.norm(b - A @ (K @ c))
    got = np.linalg.norm(b - A @ x)
    assert abs(got - best) <= 1e-9 * np.linalg.norm(b)


def test_right_preconditioning_returns_x_not_y():
    # with M^-1 = D^-1 (a diagonal scaling) the returned vector solves A x = b itself
    A, b = _system(10, 9)
    d = np.arange(1, 11, dtype=float)
    x, its, res = gm.gmres_one(A, b, lambda v: v / d, rtol=1e-12, restart=10, max_iters=10)
    assert res <= 1e-10
    assert np.allclose(A @ x, b, atol=1e-9 * np.linalg.norm(b))


def test_restarted_residuals_never_increase_between_cycles():
    # each restart cycle minimises over a space that contains the previous iterate's correction 0
    A, b = _system(40, 11)
    prev = np.inf
    for m in range(1, 6):
        _, _, res = gm.gmres_one(A, b, lambda v: v, rtol=0.0, restart=4, max_iters=4 * m)
        assert res <= prev * (1 + 1e-12)
        prev = res
