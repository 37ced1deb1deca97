"""FP32 factors with BF16 tails (hm_assemble_params.factor_tail_bits)
against the oracle.

Each block's ACA terms u_l w_l^T (Sec. 2.3) after the last one whose size
||u_l|| ||w_l|| is at least 2^-bits of the block's largest term are kept in
BF16 for the 16-right-hand-side product, the leading ones in FP32.  Checked
here: the split itself (the count of trailing terms against the same rule
applied on the host to the exported FP64 factors), the product against
oracle.hmatvec_raw on the exported operator rounded the same way (leading
terms FP32, trailing terms BF16 to nearest even, near field FP32) and
against the FP64 operator, and a batched refined solve whose inner products
run on the split copy, against the oracle's GMRES and the oracle's FP64
residual."""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu

pytestmark = pytest.mark.gpu

CASES = [
    ("ico4_leaf64", lambda: meshgen.icosphere(4), 64),
    ("bumped5_leaf128", lambda: meshgen.bump_sphere(5, 1808)[:2], 128),
]


def bf16_round64(a):
    """FP64 values rounded to the nearest BF16 (8 significant bits, ties to
    even), as FP64 (normal range only, which the factors stay in)."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)  # a = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def host_split(g, ex, bits):
    """k32 per admissible block by the rule, from the exported FP64 factors."""
    al = g.leaves(False).reshape(-1, 4)
    k32 = np.zeros(al.shape[0], dtype=np.int64)
    thr = 2.0 ** -bits
    for b in range(al.shape[0]):
        k = int(ex["rank"][b])
        if k == 0:
            continue
        m, n = al[b, 1] - al[b, 0], al[b, 3] - al[b, 2]
        U = ex["uw"][ex["u_off"][b]:ex["u_off"][b] + m * k].reshape(k, m)
        W = ex["uw"][ex["w_off"][b]:ex["w_off"][b] + n * k].reshape(k, n)
        size = np.linalg.norm(U, axis=1) * np.linalg.norm(W, axis=1)
        k32[b] = np.nonzero(size >= thr * size.max())[0].max() + 1
    return k32


def tail_rounded(g, ex, k32):
    """The exported operator as the split copy holds it."""
    al = g.leaves(False).reshape(-1, 4)
    r = dict(ex)
    r["dense"] = ex["dense"].astype(np.float32).astype(np.float64)
    uw = ex["uw"].copy()
    for b in range(al.shape[0]):
        k = int(ex["rank"][b])
        m, n = al[b, 1] - al[b, 0], al[b, 3] - al[b, 2]
        for off, rows in ((ex["u_off"][b], m), (ex["w_off"][b], n)):
            F = ex["uw"][off:off + rows * k].reshape(k, rows)
            G = np.vstack([F[:k32[b]].astype(np.float32).astype(np.float64), bf16_round64(F[k32[b]:])])
            uw[off:off + rows * k] = G.reshape(-1)
    r["uw"] = uw
    return r


def oracle_apply(orc, g, ex, X):
    perm = g.perm()
    dl, al = g.leaves(True), g.leaves(False)
    Y = np.empty_like(X)
    for r in range(X.shape[0]):
        Y[r][perm] = orc.hmatvec_raw(g.n, dl, ex["dense_off"], ex["dense"], al, ex["rank"], ex["u_off"],
                                     ex["w_off"], ex["uw"], X[r][perm])
    return Y


def test_bf16_round64_helper():
    a = np.array([1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 1.0 + 2 ** -8 + 2 ** -30])
    assert np.array_equal(bf16_round64(a), np.array([1.0, 1.0 + 2 ** -7, 1.0, 1.0 + 4 * 2 ** -8, -2.5,
                                                     1.0 + 2 ** -7]))


@pytest.mark.parametrize("name,mesh,leaf", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("bits", [8, 12])
def test_tail_product_matches_the_oracle(orc, name, mesh, leaf, bits):
    torch = need_gpu()
    V, T = mesh()
    g = GpuH(V, T, leaf=leaf, eta=1.5, eps=1e-6, factor_dtype=1, dense_dtype=1, factor_tail_bits=bits)
    try:
        hm = g.hm
        ex = g.export()
        k32 = host_split(g, ex, bits)
        host_tail = int((ex["rank"].astype(np.int64) - k32).sum())
        info = hm.hm_matrix_get_info(g.A)
        # the same rule on the same FP64 factors (sums in another order: a term
        # exactly at the threshold could fall either way)
        assert abs(info["factor_tail_terms"] - host_tail) <= 2, (info["factor_tail_terms"], host_tail)
        assert host_tail > 0.2 * ex["rank"].sum(), (host_tail, ex["rank"].sum())
        exr = tail_rounded(g, ex, k32)
        rng = np.random.default_rng(5)
        for nrhs in (16, 7):
            X = rng.standard_normal((nrhs, g.n))
            Xd = torch.from_numpy(X).cuda()
            Y = torch.empty_like(Xd)
            hm.hm_matvec_block(g.A, Xd, Y, prec=1)
            torch.cuda.synchronize()
            Yg = Y.cpu().numpy()
            ref = oracle_apply(orc, g, exr, X)
            ref64 = oracle_apply(orc, g, ex, X)
            e_copy = (np.linalg.norm(Yg - ref, axis=1) / np.linalg.norm(ref, axis=1)).max()
            e_f64 = (np.linalg.norm(Yg - ref64, axis=1) / np.linalg.norm(ref64, axis=1)).max()
            # BF16 operand pairs: ~2^-16 of the split copy's product, and the
            # trailing terms' BF16 rounding (<= 2^-(9 + bits) of a block's
            # largest term) adds little against the FP64 operator
            assert e_copy <= 3e-5, (nrhs, e_copy, e_f64)
            assert e_f64 <= 3e-5, (nrhs, e_copy, e_f64)
            # the single-right-hand-side FP32 product keeps all terms in FP32
            one = torch.empty_like(Xd[0])
            hm.hm_matvec(g.A, Xd[0].contiguous(), one, prec=1)
            torch.cuda.synchronize()
            ref32 = oracle_apply(orc, g, dict(ex, dense=exr["dense"], uw=ex["uw"].astype(np.float32)
                                              .astype(np.float64)), X[:1])[0]
            assert np.linalg.norm(one.cpu().numpy() - ref32) <= 1e-6 * np.linalg.norm(ref32)
    finally:
        g.close()


def test_tail_bits_are_checked():
    torch = need_gpu()
    import paper_1806_11558_gb300 as hm
    V, T = meshgen.icosphere(2)
    Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(T)).cuda()
    tree = hm.hm_build_tree(Vd, Td, eta=1.5, leaf_size=32)
    try:
        for bits in (-1, 1, 7, 25):
            with pytest.raises(hm.HMError) as e:
                hm.hm_assemble(tree, aca_eps=1e-6, factor_dtype=1, dense_dtype=1, factor_tail_bits=bits)
            assert e.value.status == hm.HM_EINVAL
    finally:
        hm.hm_free(tree)


def test_tail_copy_added_later_and_refined_solve(orc):
    """The split copy made by hm_matrix_add_copy after an FP64-only assembly;
    the batched refined solve on it (inner products through the split copy,
    residuals by the double-float product) reaches the oracle's FP64 residual
    and solution."""
    torch = need_gpu()
    V, T, _ = meshgen.bump_sphere(4, 1808)
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=0, dense_dtype=0, factor_tail_bits=12)
    try:
        hm = g.hm
        assert hm.hm_matrix_get_info(g.A)["factor_tail_terms"] > 0
        hm.hm_matrix_add_copy(g.A, 1)
        B = g.load_vector(meshgen.point_sources(77, 17))
        Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        Xd = torch.zeros_like(Bd)
        info = hm.hm_solve(g.A, Bd, Xd, rel_tol=1e-12, restart=60, precond=1, batched=1, max_iter=5000, refine=1,
                           inner_dtype=1, inner_tol=1e-4, max_refine=60, resid_df=1)
        torch.cuda.synchronize()
        assert info.status == 0 and info.rel_resid <= 1e-12
        X = Xd.cpu().numpy()
        perm = g.perm()
        ex = g.export()
        dl, al = g.leaves(True), g.leaves(False)

        def mv(x):
            y = np.empty(g.n)
            y[perm] = orc.hmatvec_raw(g.n, dl, ex["dense_off"], ex["dense"], al, ex["rank"], ex["u_off"],
                                      ex["w_off"], ex["uw"], x[perm])
            return y

        for r in range(B.shape[0]):
            assert np.linalg.norm(B[r] - mv(X[r])) <= 1.05e-12 * np.linalg.norm(B[r]), r
        for r in (0, 16):
            xo = orc.gmres(mv, B[r], restart=60, tol=1e-12, maxiter=20000)[0]
            assert np.linalg.norm(X[r] - xo) <= 1e-8 * np.linalg.norm(xo), r
    finally:
        g.close()
