"""Pins of the oracle's H-matrix product and GMRES."""
import numpy as np
import pytest

import meshgen


def test_gmres_matches_lu_spd(orc):
    V, T = meshgen.icosphere(3)
    A = orc.dense_matrix(V, T)
    f = orc.load_vector(V, T, [3.0, 0.0, 0.0])[0]
    x_lu = orc.lu_solve(A, f)
    x, it, rr = orc.gmres(lambda v: A @ v, f, restart=30, tol=1e-12)
    assert rr <= 1e-12
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-9


@pytest.mark.parametrize("restart", [3, 10, 30])
def test_gmres_nonsymmetric(orc, restart):
    rng = np.random.default_rng(4)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n)
    x, it, rr = orc.gmres(lambda v: A @ v, b, restart=restart, tol=1e-12, maxiter=5000)
    assert rr <= 1e-12
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-11)


def test_gmres_zero_rhs_and_maxiter(orc):
    x, it, rr = orc.gmres(lambda v: v, np.zeros(5))
    assert it == 0 and not x.any()
    A = np.diag(np.linspace(1, 1e6, 200))
    x, it, rr = orc.gmres(lambda v: A @ v, np.ones(200), restart=5, tol=1e-14, maxiter=7)
    assert it <= 7 + 5 and rr > 1e-14


@pytest.fixture(scope="module")
def level3(orc):
    V, T = meshgen.icosphere(3)
    return V, T, orc.dense_matrix(V, T)


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_hmatvec_within_10eps_of_dense(orc, level3, eps):
    V, T, A = level3
    H = orc.HMatrix(V, T, leaf=32, eta=1.5, eps=eps)
    rng = np.random.default_rng(0)
    for _ in range(3):
        x = rng.standard_normal(T.shape[0])
        assert np.linalg.norm(H.matvec(x) - A @ x) <= 10 * eps * np.linalg.norm(A @ x)
    if eps >= 1e-6:
        assert H.stored_entries() < A.size


def test_hmatvec_adjoint_and_exactness(orc, level3):
    V, T, A = level3
    H = orc.HMatrix(V, T, leaf=32, eta=1.5, eps=1e-14, kmax=200)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal((2, T.shape[0]))
    assert abs(H.matvec(x) @ y - x @ H.matvec(y, trans=True)) < 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(H.matvec(x) - A @ x) < 1e-11 * np.linalg.norm(A @ x)
    assert np.linalg.norm(H.matvec(x, trans=True) - A.T @ x) < 1e-11 * np.linalg.norm(A @ x)
