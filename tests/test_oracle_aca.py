"""Pins of the oracle's ACA with partial pivoting (Sec. 2.3)."""
import numpy as np
import pytest

import meshgen


def test_aca_rank_one_and_zero(orc):
    rng = np.random.default_rng(0)
    B = np.outer(rng.standard_normal(30), rng.standard_normal(20))
    U, W, pr, pc = orc.aca_matrix(B, 1e-12, 20)
    assert U.shape[1] in (1, 2) and np.abs(B - U @ W.T).max() < 1e-14 * np.abs(B).max()
    U, W, _, _ = orc.aca_matrix(np.zeros((5, 7)), 1e-6, 5)
    assert U.shape == (5, 0)


def test_aca_exact_low_rank_with_zero_rows(orc):
    rng = np.random.default_rng(1)
    B = rng.standard_normal((40, 6)) @ rng.standard_normal((6, 35))
    B[0] = 0.0
    B[5] = 0.0
    U, W, pr, pc = orc.aca_matrix(B, 1e-13, 30)
    assert 6 <= U.shape[1] <= 7
    assert np.abs(B - U @ W.T).max() < 1e-12 * np.abs(B).max()
    assert 0 not in pr.tolist() and len(set(pr.tolist())) == len(pr) and len(set(pc.tolist())) == len(pc)


def test_aca_interpolates_pivot_crosses(orc):
    """After k steps the residual vanishes on the chosen rows and columns."""
    x = np.linspace(0, 1, 50)
    y = np.linspace(3, 4, 45)
    B = 1.0 / np.abs(x[:, None] - y[None, :])
    for k in (1, 3, 6):
        U, W, pr, pc = orc.aca_matrix(B, 0.0, k)
        R = B - U @ W.T
        assert np.abs(R[pr, :]).max() < 1e-12 * np.abs(B).max()
        assert np.abs(R[:, pc]).max() < 1e-12 * np.abs(B).max()


def test_aca_full_rank_reproduces(orc):
    rng = np.random.default_rng(3)
    B = rng.standard_normal((12, 9))
    U, W, _, _ = orc.aca_matrix(B, 0.0, 12)
    assert U.shape[1] == 9 and np.abs(B - U @ W.T).max() < 1e-12


def test_aca_first_pivot_and_row_choice(orc):
    # first row is row 0; its largest entry picks the column, lowest index on ties
    B = np.array([[1.0, 3.0, -3.0], [2.0, 0.5, 0.1], [0.0, 4.0, 1.0]])
    U, W, pr, pc = orc.aca_matrix(B, 0.0, 1)
    assert pr.tolist() == [0] and pc.tolist() == [1]
    assert np.allclose(W[:, 0], B[0] / 3.0) and np.allclose(U[:, 0], B[:, 1])


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_aca_blocks_error_vs_dense(orc, eps):
    V, T = meshgen.icosphere(3)
    tr = orc.Tree(V, T, 32, 1.5)
    fac = orc.aca_blocks(V, T, tr.perm, tr.adm, eps, 64)
    worst = 0.0
    for (rb, re, cb, ce), (U, W) in zip(tr.adm, fac):
        B = orc.assemble(V, T, tr.perm[rb:re], tr.perm[cb:ce])
        worst = max(worst, np.linalg.norm(B - U @ W.T) / np.linalg.norm(B))
    assert worst <= 10 * eps, worst
