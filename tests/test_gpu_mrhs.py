"""Tensor-core product with many right-hand sides (hm_matvec_block) against
the oracle: the exported FP64 operator, with its near field rounded to FP32
and its factors rounded to FP32 or BF16 exactly as the library rounds its
copies (FP64 -> FP32, then -> BF16 to nearest even), applied by
oracle.hmatvec_raw one right-hand side at a time.  The tensor-core operands
are BF16 pairs (hi + lo) that keep ~16 significant bits, so the product
agrees with that reference to ~2^-16 relative; its error against the FP64
operator itself is stated as a number.  Leaves of 40, 80 and 160 rows (1,
5 and 10 row tiles of 16), 16, 5 and 20 right-hand sides (one pass, a
ragged pass, a full and a ragged pass).  Both row passes: mma.sync (the
default) and the tcgen05 / TMEM one (hm_assemble_params.mrhs_tcgen05)."""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu

pytestmark = pytest.mark.gpu

CASES = [
    ("ico4_leaf64", lambda: meshgen.icosphere(4), 64),     # leaves of 40 rows: 3 row tiles
    ("bumped5_leaf128", lambda: meshgen.bump_sphere(5, 1808)[:2], 128),  # leaves of 80 rows: 5 tiles
    ("ico3_leaf200", lambda: meshgen.icosphere(3), 200),   # leaves of 160 rows: 3 passes of 4 tiles
]


def bf16_round(a):
    """FP32 values rounded to the nearest BF16 (ties to even), as FP32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def rounded_copy(ex, prec):
    """The exported operator as the library's copies hold it."""
    r = dict(ex)
    r["dense"] = ex["dense"].astype(np.float32).astype(np.float64)
    uw32 = ex["uw"].astype(np.float32)
    r["uw"] = (uw32 if prec == 1 else bf16_round(uw32)).astype(np.float64)
    return r


def oracle_apply(orc, g, ex, X):
    perm = g.perm()
    dl, al = g.leaves(True), g.leaves(False)
    Y = np.empty_like(X)
    for r in range(X.shape[0]):
        ym = orc.hmatvec_raw(g.n, dl, ex["dense_off"], ex["dense"], al, ex["rank"], ex["u_off"], ex["w_off"],
                             ex["uw"], X[r][perm])
        Y[r][perm] = ym
    return Y


@pytest.mark.parametrize("name,mesh,leaf", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [1, 2], ids=["f32", "bf16"])
@pytest.mark.parametrize("tc", [0, 1], ids=["mma_sync", "tcgen05"])
def test_block_product_matches_the_oracle(orc, name, mesh, leaf, prec, tc):
    torch = need_gpu()
    V, T = mesh()
    g = GpuH(V, T, leaf=leaf, eta=1.5, eps=1e-6, factor_dtype=prec, dense_dtype=1, mrhs_tcgen05=tc)
    try:
        hm = g.hm
        ex = g.export()
        exr = rounded_copy(ex, prec)
        rng = np.random.default_rng(9)
        errs_copy, errs_f64 = [], []
        for nrhs in (16, 5, 20):
            X = rng.standard_normal((nrhs, g.n))
            Xd = torch.from_numpy(X).cuda()
            Y = torch.empty_like(Xd)
            hm.hm_matvec_block(g.A, Xd, Y, prec=prec)
            torch.cuda.synchronize()
            Yg = Y.cpu().numpy()
            ref = oracle_apply(orc, g, exr, X)
            ref64 = oracle_apply(orc, g, ex, X)
            e_copy = np.linalg.norm(Yg - ref, axis=1) / np.linalg.norm(ref, axis=1)
            e_f64 = np.linalg.norm(Yg - ref64, axis=1) / np.linalg.norm(ref64, axis=1)
            errs_copy.append(e_copy.max())
            errs_f64.append(e_f64.max())
            # the same copy, one right-hand side at a time on the CUDA cores (FP32 accumulation)
            one = torch.empty_like(Xd)
            for r in range(nrhs):
                hm.hm_matvec(g.A, Xd[r].contiguous(), one[r], prec=prec)
            torch.cuda.synchronize()
            e_one = np.linalg.norm(one.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
            assert e_one.max() <= 1e-6, (nrhs, e_one.max())
        # BF16 operand pairs: ~2^-16 of the copy's product
        assert max(errs_copy) <= 3e-5, (errs_copy, errs_f64)
        # against the FP64 operator: the copy's own rounding on top (FP32 entries 6e-8, BF16 factors 2^-9)
        assert max(errs_f64) <= (3e-5 if prec == 1 else 4e-3), (errs_copy, errs_f64)
        # alpha, beta
        X = torch.from_numpy(rng.standard_normal((3, g.n))).cuda()
        Y0 = torch.from_numpy(rng.standard_normal((3, g.n))).cuda()
        Y = Y0.clone()
        hm.hm_matvec_block(g.A, X, Y, prec=prec, alpha=2.0, beta=-0.5)
        ref = torch.empty_like(X)
        hm.hm_matvec_block(g.A, X, ref, prec=prec)
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(Y - (2.0 * ref - 0.5 * Y0))) <= 1e-12 * float(torch.linalg.norm(Y))
    finally:
        g.close()


def test_bf16_rounding_helper():
    # exact BF16 values stay; halfway cases go to the even neighbour
    a = np.array([1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5], dtype=np.float32)
    assert np.array_equal(bf16_round(a), np.array([1.0, 1.0 + 2 ** -7, 1.0, 1.0 + 4 * 2 ** -8, -2.5],
                                                  dtype=np.float32))


def test_block_product_rejects_unknown_precision_and_missing_copies():
    torch = need_gpu()
    V, T = meshgen.icosphere(2)
    g = GpuH(V, T, eps=1e-6, factor_dtype=0, dense_dtype=0)
    try:
        x = torch.zeros((2, g.n), dtype=torch.float64, device="cuda")
        for prec in (3, -1):
            with pytest.raises(g.hm.HMError) as e:
                g.hm.hm_matvec_block(g.A, x, x.clone(), prec=prec)
            assert e.value.status == g.hm.HM_EINVAL
        for prec in (1, 2):  # no FP32 / BF16 copies assembled
            with pytest.raises(g.hm.HMError) as e:
                g.hm.hm_matvec_block(g.A, x, x.clone(), prec=prec)
            assert e.value.status == g.hm.HM_EINVAL
    finally:
        g.close()
