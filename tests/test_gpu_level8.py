"""GPU path vs the oracle at the size bench.py times: the unit icosphere of
level 8 (1,310,720 panels), C_leaf = 128 (leaf clusters of 80 panels),
eta = 1.5, ACA eps = 1e-6, 16 point sources, with the FP32 copies of the near
field and the factors beside the FP64 master (the configuration of the
timed step) and the BF16 factors added from the master.

The oracle cannot assemble this matrix in a test's time, so the checks are:
the integer stage in full (bit-exact); sampled near-field entries; every
admissible size class against the oracle's dense block (whole blocks up to
5,120 x 5,120, which covers the ACA's tier for m + n > 2,560, and single
columns of the blocks of 10,240 .. 81,920 rows: inside a leaf block,
(H e_j) restricted to the block's rows is exactly column j of that block);
sampled rows of the one- and 16-right-hand-side products against rows of the
Galerkin matrix computed by the oracle; the load vectors; and the mixed
solution of two of the systems against the FP64 one.  Tolerances: ACA blocks
10 eps (Frobenius, as in test_gpu_parity.py); product rows 10 eps |A||x|
plus, for the tensor-core product, the BF16 operand pairs (2^-16 of |A||x|).
"""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu, split_dense_rows

pytestmark = pytest.mark.gpu

EPS = 1e-6
LEAF = 128


def _sorted(a):
    a = np.asarray(a, dtype=np.int64).reshape(-1, 4)
    return a[np.lexsort(a.T[::-1])]


@pytest.fixture(scope="module")
def big(orc):
    need_gpu()
    cfg = meshgen.config("large")
    V, T = cfg["V"], cfg["T"]
    g = GpuH(V, T, leaf=LEAF, eta=1.5, eps=EPS, kmax=64, ss_order=8, factor_dtype=1, dense_dtype=1)
    g.hm.hm_matrix_add_copy(g.A, g.hm.HM_BF16)
    tr = orc.Tree(V, T, LEAF, 1.5)
    yield g, tr, cfg
    g.close()


def test_level8_tree_bit_exact(big):
    g, tr, _ = big
    assert g.n == 1310720
    assert np.array_equal(g.perm(), tr.perm)
    assert np.array_equal(_sorted(g.leaves(False)), _sorted(tr.adm))
    assert np.array_equal(_sorted(g.leaves(True)), _sorted(split_dense_rows(tr.dense, LEAF)))


def test_level8_sampled_entries(orc, big):
    g, tr, _ = big
    perm = g.perm()
    rng = np.random.default_rng(11)
    dense = g.leaves(True)
    worst_reg = worst_sing = 0.0
    for b in rng.choice(len(dense), size=300, replace=False):
        rb, re, cb, ce = dense[b]
        blk = g.block(True, b, dense[b])
        for _ in range(5):
            i, j = int(rng.integers(re - rb)), int(rng.integers(ce - cb))
            ref = orc.entry(g.V, g.T, perm[rb + i], perm[cb + j])
            rel = abs(blk[i, j] - ref) / abs(ref)
            if orc.touch(g.T, perm[rb + i], perm[cb + j]):
                worst_sing = max(worst_sing, rel)
            else:
                worst_reg = max(worst_reg, rel)
    assert worst_reg < 1e-13 and worst_sing < 1e-12, (worst_reg, worst_sing)


def test_level8_admissible_blocks_every_size_class(orc, big):
    g, tr, _ = big
    torch = g.torch
    perm = g.perm()
    rng = np.random.default_rng(12)
    adm = g.leaves(False)
    sizes = adm[:, 1] - adm[:, 0]
    classes = np.unique(sizes)
    assert classes.max() == 81920  # the largest admissible blocks of this mesh
    worst = {}
    for sz in classes:
        idx = np.flatnonzero(sizes == sz)
        if sz <= 5120:
            # whole blocks: up to 1,280 (warp and CTA workers) and the huge tier (m + n > 2,560)
            for b in rng.choice(idx, size=min(2, len(idx)), replace=False):
                rb, re, cb, ce = adm[b]
                B = orc.assemble(g.V, g.T, perm[rb:re], perm[cb:ce])
                err = np.linalg.norm(B - g.block(False, b, adm[b])) / np.linalg.norm(B)
                worst[int(sz)] = max(worst.get(int(sz), 0.0), err)
        else:
            # single columns of one block above and one below the diagonal
            upper = idx[adm[idx, 0] < adm[idx, 2]]
            lower = idx[adm[idx, 0] > adm[idx, 2]]
            for pool in (upper, lower):
                if len(pool) == 0:
                    continue
                b = int(rng.choice(pool))
                rb, re, cb, ce = adm[b]
                cols = rng.choice(np.arange(cb, ce), size=3, replace=False)
                E = torch.zeros((3, g.n), dtype=torch.float64, device="cuda")
                for r, j in enumerate(cols):
                    E[r, int(perm[j])] = 1.0
                Y = torch.empty_like(E)
                g.hm.hm_matvec(g.A, E, Y)
                torch.cuda.synchronize()
                Yh = Y.cpu().numpy()
                for r, j in enumerate(cols):
                    col = Yh[r][perm[rb:re]]
                    ref = orc.assemble(g.V, g.T, perm[rb:re], [perm[j]])[:, 0]
                    err = np.linalg.norm(col - ref) / np.linalg.norm(ref)
                    worst[int(sz)] = max(worst.get(int(sz), 0.0), err)
    assert len(worst) == len(classes)
    assert max(worst.values()) <= 10 * EPS, worst


def test_level8_sampled_rows_of_the_products(orc, big):
    g, tr, _ = big
    torch, hm = g.torch, g.hm
    rng = np.random.default_rng(13)
    X = rng.standard_normal((16, g.n))
    rows = rng.choice(g.n, size=16, replace=False)
    A_rows = orc.assemble(g.V, g.T, rows, np.arange(g.n))
    ref = A_rows @ X.T            # [16 rows, 16 rhs]
    scale = np.abs(A_rows) @ np.abs(X.T)
    Xd = torch.from_numpy(X).cuda()
    Y = torch.empty_like(Xd)
    got = {}
    # one right-hand side on the FP64 master, 16 at a time on the tensor cores (FP32 and BF16 factors)
    hm.hm_matvec(g.A, Xd, Y)
    torch.cuda.synchronize()
    got["fp64"] = Y.cpu().numpy()[:, rows].T
    for name, prec in (("16rhs_fp32", hm.HM_F32), ("16rhs_bf16", hm.HM_BF16)):
        hm.hm_matvec_block(g.A, Xd, Y, prec=prec)
        torch.cuda.synchronize()
        got[name] = Y.cpu().numpy()[:, rows].T
    ratio = {k: float(np.max(np.abs(v - ref) / scale)) for k, v in got.items()}
    assert ratio["fp64"] <= 10 * EPS, ratio
    # BF16 operand pairs keep ~16 bits (2^-16 = 1.5e-5 of |A||x|) on top of the ACA error
    assert ratio["16rhs_fp32"] <= 10 * EPS + 3e-5, ratio
    assert ratio["16rhs_bf16"] <= 10 * EPS + 3e-5 + 2 ** -8, ratio


def test_level8_load_vectors_and_mixed_solution(orc, big):
    g, tr, cfg = big
    torch, hm = g.torch, g.hm
    src = cfg["sources"][:2]
    F = g.load_vector(src)
    pick = np.random.default_rng(14).choice(g.n, size=200, replace=False)
    Fo = orc.load_vector(g.V, g.T[pick], src)
    assert np.abs(F[:, pick] - Fo).max() <= 1e-14 * np.abs(Fo).max()
    opts = dict(rel_tol=1e-12, restart=128, max_iter=5000, precond=1, batched=1)
    X64, i64 = g.solve(F, **opts)
    Xm, im = g.solve(F, refine=1, inner_dtype=hm.HM_F32, inner_tol=1e-4, max_refine=40, **opts)
    assert i64.status == 0 and i64.rel_resid <= 1e-12
    assert im.status == 0 and im.rel_resid <= 1e-12 and im.refine_steps >= 1
    err = np.linalg.norm(Xm - X64, axis=1) / np.linalg.norm(X64, axis=1)
    assert err.max() < 1e-8, err
    # the FP64 residual of the mixed solution, recomputed through the product
    for r in range(2):
        res = F[r] - g.matvec(Xm[r])
        assert np.linalg.norm(res) <= 1.01e-12 * np.linalg.norm(F[r])
