"""GPU path vs the oracle at the benchmark's workload size: the bumped
icosphere of level 7 (327,680 panels), C_leaf = 64, eta = 1.5, ACA eps = 1e-7,
in the configuration bench.py times.

The oracle cannot assemble this matrix in a test's time budget, so the
checks are: the integer stage in full (bit-exact); sampled near-field
entries, sampled admissible blocks and sampled rows of the product, each
computed by the oracle one by one; and properties that hold at any size
(residuals of the solves, mixed precision against FP64).  Tolerances as in
test_gpu_parity.py.
"""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, as_set, need_gpu, split_dense_rows

pytestmark = pytest.mark.gpu

EPS = 1e-7


@pytest.fixture(scope="module")
def big(orc):
    need_gpu()
    cfg = meshgen.config("precision")
    V, T = cfg["V"], cfg["T"]
    g = GpuH(V, T, leaf=64, eta=1.5, eps=EPS, kmax=64, ss_order=8, factor_dtype=1, dense_dtype=1)
    tr = orc.Tree(V, T, 64, 1.5)
    yield g, tr
    g.close()


def test_fullsize_tree_bit_exact(big):
    g, tr = big
    assert np.array_equal(g.perm(), tr.perm)
    assert as_set(g.leaves(False)) == as_set(tr.adm)
    assert as_set(g.leaves(True)) == as_set(split_dense_rows(tr.dense, 64))


def test_fullsize_sampled_entries_and_blocks(orc, big):
    g, tr = big
    perm = g.perm()
    rng = np.random.default_rng(7)
    # near field: 2000 random entries of random dense leaves
    dense = g.leaves(True)
    worst_reg = worst_sing = 0.0
    for b in rng.choice(len(dense), size=400, replace=False):
        rb, re, cb, ce = dense[b]
        m, n = re - rb, ce - cb
        blk = g.block(True, b, dense[b])
        for _ in range(5):
            i, j = int(rng.integers(m)), int(rng.integers(n))
            ref = orc.entry(g.V, g.T, perm[rb + i], perm[cb + j])
            rel = abs(blk[i, j] - ref) / abs(ref)
            if orc.touch(g.T, perm[rb + i], perm[cb + j]):
                worst_sing = max(worst_sing, rel)
            else:
                worst_reg = max(worst_reg, rel)
    assert worst_reg < 1e-13 and worst_sing < 1e-12, (worst_reg, worst_sing)
    # admissible blocks: every size class, against the oracle's dense block
    adm = g.leaves(False)
    sizes = adm[:, 1] - adm[:, 0]
    picks = []
    for sz in np.unique(sizes):
        if sz > 1280:
            continue
        idx = np.flatnonzero(sizes == sz)
        picks += list(rng.choice(idx, size=min(3, len(idx)), replace=False))
    worst = 0.0
    for b in picks:
        rb, re, cb, ce = adm[b]
        B = orc.assemble(g.V, g.T, perm[rb:re], perm[cb:ce])
        worst = max(worst, np.linalg.norm(B - g.block(False, b, adm[b])) / np.linalg.norm(B))
    assert worst <= 10 * EPS, worst


def test_fullsize_sampled_matvec_rows(orc, big):
    g, tr = big
    rng = np.random.default_rng(3)
    x = rng.standard_normal(g.n)
    y = g.matvec(x)
    rows = rng.choice(g.n, size=24, replace=False)
    A_rows = orc.assemble(g.V, g.T, rows, np.arange(g.n))
    yo = A_rows @ x
    # each sampled row within 10 eps of the row of A times |x| (entry-wise bound of the block errors)
    scale = np.abs(A_rows) @ np.abs(x)
    assert np.all(np.abs(y[rows] - yo) <= 10 * EPS * scale), np.max(np.abs(y[rows] - yo) / scale)
    y32 = g.matvec(x, prec=1)
    assert np.linalg.norm(y32 - y) <= 1e-5 * np.linalg.norm(y)


def test_fullsize_load_vector_and_solves(orc, big):
    g, tr = big
    src = np.array([3.0, 0.0, 0.0])
    f = g.load_vector(src)[0]
    rng = np.random.default_rng(5)
    pick = rng.choice(g.n, size=200, replace=False)
    fo = orc.load_vector(g.V, g.T[pick], src)[0]
    assert np.abs(f[pick] - fo).max() <= 1e-14 * np.abs(fo).max()
    x64, i64 = g.solve(f, rel_tol=1e-12, precond=1, max_iter=5000)
    assert i64.status == 0 and i64.rel_resid <= 1e-12
    xm, im = g.solve(f, rel_tol=1e-12, precond=1, refine=1, inner_tol=1e-4, inner_dtype=1, max_iter=5000)
    assert im.rel_resid <= 1e-12
    assert np.linalg.norm(xm - x64) / np.linalg.norm(x64) < 1e-8
    # the FP64 residual of the solution, recomputed through the product
    r = f - g.matvec(x64)
    assert np.linalg.norm(r) <= 1.01e-12 * np.linalg.norm(f)
