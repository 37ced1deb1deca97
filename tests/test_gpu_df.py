"""The 16-right-hand-side product of the FP64 master in double-float
arithmetic (hm_matvec_block with HM_F64) against the oracle: the exported
FP64 operator applied by oracle.hmatvec_raw in FP64, one right-hand side at
a time.  Every entry and x are split into pairs of floats (w = h + l up to
2^-47 |w|) and each term is accumulated with an error-free product and sum
(the compensated dot product of Ogita, Rump and Oishi), so each row of the
result is within a few units of 2^-47 of the row sum of |H||x| plus the
rounding of the float compensation, about sqrt(n) u^2 of it for the n
terms of one accumulator (u = 2^-24; n up to ~600 here: ~9e-14): the bound
asserted is 2e-13 of that row sum, row by row, and 2e-14 of the norm of the
row sums (random right-hand sides cancel: ||H x|| itself is an order or two
below it).  Leaves
of 40, 80 and 160 rows (the three shapes of the row pass, the last in two
tiles), 16, 5 and 20 right-hand sides; a mesh scaled by 1e-5, whose entries
span the range where the split leaves the integer path; alpha / beta."""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu

pytestmark = pytest.mark.gpu

CASES = [
    ("ico4_leaf64", lambda: meshgen.icosphere(4), 64),
    ("bumped5_leaf128", lambda: meshgen.bump_sphere(5, 1808)[:2], 128),
    ("ico3_leaf200", lambda: meshgen.icosphere(3), 200),
    ("ico3_scaled_1e-5", lambda: (meshgen.icosphere(3)[0] * 1e-5, meshgen.icosphere(3)[1]), 64),
]


def oracle_apply(orc, g, ex, X):
    perm = g.perm()
    dl, al = g.leaves(True), g.leaves(False)
    Y = np.empty_like(X)
    for r in range(X.shape[0]):
        Y[r][perm] = orc.hmatvec_raw(g.n, dl, ex["dense_off"], ex["dense"], al, ex["rank"], ex["u_off"],
                                     ex["w_off"], ex["uw"], X[r][perm])
    return Y


def abs_operator(ex):
    """|H| entrywise on the stored form: |D| and, for the factors, |U| |W|^T (>= |U W^T|)."""
    r = dict(ex)
    r["dense"] = np.abs(ex["dense"])
    r["uw"] = np.abs(ex["uw"])
    return r


@pytest.mark.parametrize("name,mesh,leaf", CASES, ids=[c[0] for c in CASES])
def test_double_float_product_matches_the_oracle(orc, name, mesh, leaf):
    torch = need_gpu()
    V, T = mesh()
    g = GpuH(V, T, leaf=leaf, eta=1.5, eps=1e-8, factor_dtype=0, dense_dtype=0)
    try:
        hm = g.hm
        ex = g.export()
        exa = abs_operator(ex)
        rng = np.random.default_rng(21)
        for nrhs in (16, 5, 20):
            X = rng.standard_normal((nrhs, g.n))
            Xd = torch.from_numpy(X).cuda()
            Y = torch.empty_like(Xd)
            hm.hm_matvec_block(g.A, Xd, Y, prec=hm.HM_F64)
            torch.cuda.synchronize()
            Yg = Y.cpu().numpy()
            ref = oracle_apply(orc, g, ex, X)
            mag = oracle_apply(orc, g, exa, np.abs(X))  # row sums of |H||x| (an upper bound)
            rows = np.abs(Yg - ref) / mag
            e = np.linalg.norm(Yg - ref, axis=1) / np.linalg.norm(mag, axis=1)
            assert rows.max() <= 2e-13 and e.max() <= 2e-14, (nrhs, rows.max(), e.max())
        # alpha, beta
        X = torch.from_numpy(rng.standard_normal((3, g.n))).cuda()
        Y0 = torch.from_numpy(rng.standard_normal((3, g.n))).cuda()
        Y = Y0.clone()
        hm.hm_matvec_block(g.A, X, Y, prec=hm.HM_F64, alpha=2.0, beta=-0.5)
        ref = torch.empty_like(X)
        hm.hm_matvec_block(g.A, X, ref, prec=hm.HM_F64)
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(Y - (2.0 * ref - 0.5 * Y0))) <= 1e-12 * float(torch.linalg.norm(Y))
    finally:
        g.close()


def test_double_float_product_of_zeros_and_one_column(orc):
    torch = need_gpu()
    V, T = meshgen.icosphere(3)
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=0, dense_dtype=0)
    try:
        hm = g.hm
        X = torch.zeros((16, g.n), dtype=torch.float64, device="cuda")
        Y = torch.full_like(X, 7.0)
        hm.hm_matvec_block(g.A, X, Y, prec=hm.HM_F64)
        torch.cuda.synchronize()
        assert torch.count_nonzero(Y) == 0
        # a unit vector: the column of H, against the oracle's product
        x = np.zeros((1, g.n))
        x[0, g.n // 3] = 1.0
        y = torch.empty((1, g.n), dtype=torch.float64, device="cuda")
        hm.hm_matvec_block(g.A, torch.from_numpy(x).cuda(), y, prec=hm.HM_F64)
        torch.cuda.synchronize()
        ex = g.export()
        ref = oracle_apply(orc, g, ex, x)
        mag = oracle_apply(orc, g, abs_operator(ex), np.abs(x))
        assert np.all(np.abs(y.cpu().numpy() - ref) <= 2e-13 * mag)
    finally:
        g.close()
