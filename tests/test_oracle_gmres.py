"""Pins of the oracle's restarted, left-preconditioned GMRES (Sec. 4)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.gmres import givens, gmres


def _spd(n, rng):
    X = rng.standard_normal((n, n))
    return X @ X.T + n * np.eye(n)


def _csym(n, rng):
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return X + X.T + 2 * n * np.eye(n)


@pytest.mark.parametrize("kind", ["spd", "csym"])
def test_matches_direct_solve(kind):
    rng = np.random.default_rng(1)
    n = 60
    A = _spd(n, rng) if kind == "spd" else _csym(n, rng)
    b = rng.standard_normal(n) + (1j * rng.standard_normal(n) if kind == "csym" else 0)
    d = np.diag(A)
    r = gmres(A, b, lambda v: v / d, tol=1e-12, restart=10, maxit=500)
    assert r.converged
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(r.x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_exact_after_n_steps():
    """Full GMRES (n <= restart) terminates with the exact solution by step n."""
    rng = np.random.default_rng(2)
    n = 12
    A = rng.standard_normal((n, n)) + 3 * np.eye(n)
    b = rng.standard_normal(n)
    r = gmres(A, b, lambda v: v, tol=1e-13, restart=30, maxit=30)
    assert r.converged and r.iters <= n
    assert np.linalg.norm(A @ r.x - b) <= 1e-11 * np.linalg.norm(b)


def test_residual_monotone_within_cycle():
    rng = np.random.default_rng(3)
    n = 80
    A = sp.random(n, n, density=0.1, random_state=3) + 4 * sp.eye(n)
    A = A.tocsr()
    b = rng.standard_normal(n)
    r = gmres(A, b, lambda v: v, tol=1e-10, restart=30, maxit=30)
    h = np.array(r.history)
    assert np.all(np.diff(h) <= 1e-14 * h[0])


def test_exact_preconditioner_one_step():
    rng = np.random.default_rng(4)
    A = _csym(30, rng)
    b = rng.standard_normal(30).astype(complex)
    Ai = np.linalg.inv(A)
    r = gmres(A, b, lambda v: Ai @ v)
    assert r.converged and r.iters == 1


def test_givens_zeroes_second_component():
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, b = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        c, s = givens(a, b)
        assert abs(-np.conj(s) * a + c * b) <= 1e-15 * (abs(a) + abs(b))
        assert abs(abs(c) ** 2 + abs(s) ** 2 - 1) <= 1e-15
