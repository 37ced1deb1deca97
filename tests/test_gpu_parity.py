"""GPU path vs the oracle, element by element, on small meshes.

Tolerances: integer stage bit-exact.  Regular entries are 49 positive terms
of w_p w_q / r with r from the same quadrature points (the GPU computes the
points with the same rounded operations) but rsqrt / fma instead of the
oracle's 1/sqrt and separate multiply-add: a few ulp, bound 1e-13 relative.
Touching pairs sum up to 6 * 8^3 positive terms in another order: bound
1e-12 relative.  ACA blocks: ||B - U W^T||_F <= 10 eps ||B||_F (the pivots
may differ from the oracle's on near ties, so factors are not compared
entry-wise).  H-matvec: within 10 eps of the dense product; the GPU product
and the oracle's re-application of the exported GPU H-matrix agree to 1e-12.
"""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, as_set, need_gpu, split_dense_rows

pytestmark = pytest.mark.gpu


def _meshes():
    out = {}
    out["ico3"] = meshgen.icosphere(3)
    out["ico4"] = meshgen.icosphere(4)
    V, T, _ = meshgen.bump_sphere(3, 1808)
    out["bump3"] = (V, T)
    out["stretch3"] = (meshgen.stretch(meshgen.icosphere(3)[0], [2.0, 0.7, 1.3]), meshgen.icosphere(3)[1])
    V, T = meshgen.icosphere(3)
    out["open1000"] = (V, np.ascontiguousarray(T[:1000]))  # ragged N, open surface
    return out


MESHES = _meshes()


@pytest.mark.parametrize("name,leaf,eta", [("ico3", 64, 1.5), ("ico4", 64, 1.5), ("bump3", 16, 1.0),
                                           ("stretch3", 32, 1.5), ("open1000", 64, 1.5), ("open1000", 7, 2.0),
                                           ("ico3", 1, 1.5)])
def test_tree_bit_exact(orc, name, leaf, eta):
    need_gpu()
    V, T = MESHES[name]
    tr = orc.Tree(V, T, leaf, eta)
    g = GpuH(V, T, leaf=leaf, eta=eta, eps=None)
    try:
        assert np.array_equal(g.perm(), tr.perm)
        assert as_set(g.leaves(False)) == as_set(tr.adm)
        assert as_set(g.leaves(True)) == as_set(split_dense_rows(tr.dense, leaf))
        info = g.info()
        assert info["n_adm"] == len(tr.adm)
        assert info["adm_rows_cols"] == int(((tr.adm[:, 1] - tr.adm[:, 0]) + (tr.adm[:, 3] - tr.adm[:, 2])).sum())
    finally:
        g.close()


@pytest.fixture(scope="module")
def ico3(orc):
    need_gpu()
    V, T = MESHES["ico3"]
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=1, dense_dtype=1)
    A = orc.dense_matrix(V, T)
    yield g, A
    g.close()


def _nearfield_errors(orc, g, A):
    perm = g.perm()
    ex = g.export()
    dense = g.leaves(True)
    worst_reg = worst_sing = 0.0
    n_vertex = n_other = 0
    for b, (rb, re, cb, ce) in enumerate(dense):
        m, n = re - rb, ce - cb
        blk = ex["dense"][ex["dense_off"][b]:ex["dense_off"][b] + m * n].reshape(m, n)
        ref = A[np.ix_(perm[rb:re], perm[cb:ce])]
        rel = np.abs(blk - ref) / np.abs(ref)
        kind = np.array([[orc.touch(g.T, perm[rb + i], perm[cb + j]) for j in range(n)] for i in range(m)])
        touch = kind > 0
        n_vertex += int((kind == 1).sum())
        n_other += int((kind > 1).sum())
        if (~touch).any():
            worst_reg = max(worst_reg, rel[~touch].max())
        if touch.any():
            worst_sing = max(worst_sing, rel[touch].max())
    return worst_reg, worst_sing, n_vertex, n_other


def test_nearfield_entries(orc, ico3):
    # regular entries in double-float arithmetic (the default)
    g, A = ico3
    worst_reg, worst_sing, n_vertex, n_other = _nearfield_errors(orc, g, A)
    assert worst_reg < 1e-13, worst_reg
    assert worst_sing < 1e-12, worst_sing
    # every dense leaf here is diagonal or has its transposed partner: a
    # common-vertex pair is evaluated once for both positions, edge and
    # identical pairs once per position
    assert n_vertex % 2 == 0
    assert g.info()["n_singular"] == n_other + n_vertex // 2


def test_nearfield_entries_fp64_arithmetic(orc, ico3):
    # the same entries with FP64 arithmetic; touching pairs are unchanged
    g0, A = ico3
    V, T = MESHES["ico3"]
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, nearfield_fp64=1)
    try:
        worst_reg, worst_sing, _, _ = _nearfield_errors(orc, g, A)
        assert worst_reg < 1e-13, worst_reg
        assert worst_sing < 1e-12, worst_sing
    finally:
        g.close()


def test_aca_blocks_within_tolerance(orc, ico3):
    g, A = ico3
    perm = g.perm()
    ex = g.export()
    adm = g.leaves(False)
    worst = 0.0
    for b, (rb, re, cb, ce) in enumerate(adm):
        m, n, k = re - rb, ce - cb, ex["rank"][b]
        U = ex["uw"][ex["u_off"][b]:ex["u_off"][b] + m * k].reshape(k, m).T
        W = ex["uw"][ex["w_off"][b]:ex["w_off"][b] + n * k].reshape(k, n).T
        B = A[np.ix_(perm[rb:re], perm[cb:ce])]
        worst = max(worst, np.linalg.norm(B - U @ W.T) / np.linalg.norm(B))
    assert worst <= 10 * 1e-8, worst


def test_matvec_vs_dense_and_same_operator(orc, ico3):
    g, A = ico3
    rng = np.random.default_rng(0)
    perm = g.perm()
    ex = g.export()
    ti = g.info()
    for _ in range(3):
        x = rng.standard_normal(g.n)
        y = g.matvec(x)
        assert np.linalg.norm(y - A @ x) <= 10 * 1e-8 * np.linalg.norm(A @ x)
        # oracle re-application of the exported GPU H-matrix (Morton order)
        ym = orc.hmatvec_raw(g.n, g.leaves(True), ex["dense_off"], ex["dense"], g.leaves(False), ex["rank"],
                             ex["u_off"], ex["w_off"], ex["uw"], x[perm])
        yo = np.empty(g.n)
        yo[perm] = ym
        assert np.linalg.norm(y - yo) <= 1e-12 * np.linalg.norm(yo)
        # FP32 copy: within single-precision accuracy of the FP64 product
        y32 = g.matvec(x, prec=1)
        assert np.linalg.norm(y32 - y) <= 1e-5 * np.linalg.norm(y)
    assert ti["n_dense"] > 0 and ti["n_adm"] > 0


def test_load_vector(orc, ico3):
    g, _ = ico3
    src = np.array([[3.0, 0.0, 0.0], [0.5, -2.2, 1.7]])
    f = g.load_vector(src)
    fo = orc.load_vector(g.V, g.T, src)
    assert np.abs(f - fo).max() <= 1e-14 * np.abs(fo).max()


def test_solve_fp64_and_mixed(orc, ico3):
    g, A = ico3
    f = orc.load_vector(g.V, g.T, [3.0, 0.0, 0.0])[0]
    x64, info = g.solve(f, rel_tol=1e-12)
    assert info.rel_resid <= 1e-12 and info.status == 0
    x_lu = orc.lu_solve(A, f)
    # H at eps = 1e-8 differs from A by ~1e-8: solution within a small multiple of kappa * eps
    assert np.linalg.norm(x64 - x_lu) / np.linalg.norm(x_lu) < 1e-6
    # the same operator solved by the oracle's GMRES on the exported H-matrix
    perm = g.perm()
    ex = g.export()
    dl, al = g.leaves(True), g.leaves(False)

    def mv(x):
        ym = orc.hmatvec_raw(g.n, dl, ex["dense_off"], ex["dense"], al, ex["rank"], ex["u_off"], ex["w_off"],
                             ex["uw"], x[perm])
        y = np.empty(g.n)
        y[perm] = ym
        return y

    xo, it, rr = orc.gmres(mv, f, restart=30, tol=1e-12)
    assert np.linalg.norm(x64 - xo) / np.linalg.norm(xo) < 1e-8
    xm, im = g.solve(f, rel_tol=1e-12, refine=1, inner_tol=1e-4, inner_dtype=1)
    assert im.rel_resid <= 1e-12 and im.refine_steps >= 1
    assert np.linalg.norm(xm - x64) / np.linalg.norm(x64) < 1e-8
    # block-Jacobi right preconditioning: same operator, same solution, fewer steps
    xp, ip = g.solve(f, rel_tol=1e-12, precond=1)
    assert ip.rel_resid <= 1e-12 and ip.iters < info.iters
    assert np.linalg.norm(xp - xo) / np.linalg.norm(xo) < 1e-8
    xpm, ipm = g.solve(f, rel_tol=1e-12, refine=1, inner_tol=1e-4, inner_dtype=1, precond=1)
    assert ipm.rel_resid <= 1e-12
    assert np.linalg.norm(xpm - xo) / np.linalg.norm(xo) < 1e-8


def test_solve_dense_limit_matches_lu(orc):
    """eps -> 0: the H-matrix reproduces A and the solution reaches the LU one."""
    need_gpu()
    V, T = MESHES["ico3"]
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-13, kmax=128)
    try:
        A = orc.dense_matrix(V, T)
        f = orc.load_vector(V, T, [3.0, 0.0, 0.0])[0]
        x, info = g.solve(f, rel_tol=1e-13)
        x_lu = orc.lu_solve(A, f)
        assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-8
    finally:
        g.close()


def test_bf16_factors_refined_to_fp64_accuracy(orc):
    need_gpu()
    V, T = MESHES["bump3"]
    g = GpuH(V, T, leaf=32, eta=1.5, eps=1e-7, factor_dtype=2, dense_dtype=1)
    try:
        f = orc.load_vector(V, T, [3.0, 0.0, 0.0])[0]
        x64, _ = g.solve(f, rel_tol=1e-12)
        xb, ib = g.solve(f, rel_tol=1e-12, refine=1, inner_tol=1e-2, inner_dtype=2, max_refine=40)
        assert ib.rel_resid <= 1e-12
        assert np.linalg.norm(xb - x64) / np.linalg.norm(x64) < 1e-8
    finally:
        g.close()


@pytest.mark.parametrize("case", ["one", "edge_pair", "vertex_pair", "strip"])
def test_degenerate_meshes(orc, case):
    need_gpu()
    if case == "one":
        V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
        T = np.array([[0, 1, 2]], dtype=np.int32)
    elif case == "edge_pair":
        V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0.3]])
        T = np.array([[0, 1, 2], [2, 1, 3]], dtype=np.int32)
    elif case == "vertex_pair":
        V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0.2], [0, -1, 0.1]])
        T = np.array([[0, 1, 2], [0, 3, 4]], dtype=np.int32)
    else:
        V, T = meshgen.icosphere(2)
        T = np.ascontiguousarray(T[:37])
    g = GpuH(V, T, leaf=4, eta=1.5, eps=1e-10, factor_dtype=1, dense_dtype=1)
    try:
        A = orc.dense_matrix(V, T)
        x = np.linspace(1.0, 2.0, T.shape[0])
        y = g.matvec(x)
        assert np.linalg.norm(y - A @ x) <= 1e-9 * np.linalg.norm(A @ x)
        # preconditioned solve in its graph form, and the 16-right-hand-side
        # product, on the same degenerate trees
        xs, info = g.solve(A @ x, rel_tol=1e-12, restart=30, precond=1, use_graph=1, max_iter=500)
        assert info.status == 0
        assert np.linalg.norm(xs - x) <= 1e-8 * np.linalg.norm(x)
        torch = g.torch
        X = np.stack([x, x[::-1].copy(), np.ones_like(x)])
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        Yd = torch.empty_like(Xd)
        g.hm.hm_matvec_block(g.A, Xd, Yd, prec=1)
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy()
        for r in range(3):
            assert np.linalg.norm(Y[r] - A @ X[r]) <= 1e-4 * np.linalg.norm(A @ X[r])
    finally:
        g.close()


def test_kappa_estimate_from_hessenberg(orc):
    # sigma_max / sigma_min of the first cycle's Hessenberg factor lies inside
    # the operator's condition number and, with a Krylov space long enough to
    # converge, close to it (the spectrum's ends converge first); the
    # reference is the dense oracle matrix's eigenvalue ratio (it is SPD)
    need_gpu()
    V, T = MESHES["ico3"]
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-12, kmax=128)
    try:
        A = orc.dense_matrix(V, T)
        ev = np.linalg.eigvalsh(0.5 * (A + A.T))
        kappa = ev[-1] / ev[0]
        b = g.load_vector(np.array([[3.0, 0.0, 0.0]]))[0]
        x, info = g.solve(b, rel_tol=1e-12, restart=128, max_iter=128, raise_on_noconv=False)
        assert info.restarts == 1 and info.iters >= 40
        assert 0.7 * kappa <= info.kappa_est <= 1.001 * kappa, (info.kappa_est, kappa)
        # refined and preconditioned solves report the estimate of their operator
        _, ip = g.solve(b, rel_tol=1e-12, restart=128, max_iter=500, precond=1)
        assert 1.0 <= ip.kappa_est < kappa
    finally:
        g.close()


def test_wide_leaves_use_the_fp64_fallbacks(orc):
    # 1,016 panels with leaf 254: leaf clusters of 254 panels, wider than the
    # float-pair staging box (250) and the shared-memory block inversion
    # (232), so the FP64 near-field kernel and the FP64 global-memory
    # block-Jacobi inversion run; both against the oracle
    need_gpu()
    V, T = meshgen.icosphere(3)
    T = np.ascontiguousarray(T[:1016])
    g = GpuH(V, T, leaf=254, eta=1.5, eps=1e-10, kmax=128)
    try:
        assert g.info()["max_leaf"] == 254
        A = orc.dense_matrix(V, T)
        worst_reg, worst_sing, _, _ = _nearfield_errors(orc, g, A)
        assert worst_reg < 1e-13 and worst_sing < 1e-12, (worst_reg, worst_sing)
        b = g.load_vector(np.array([[3.0, 0.0, 0.0]]))[0]
        x, info = g.solve(b, rel_tol=1e-12, restart=60, precond=1, max_iter=2000)
        assert info.status == 0
        x_lu = np.linalg.solve(A, b)
        assert np.linalg.norm(x - x_lu) <= 1e-7 * np.linalg.norm(x_lu)
    finally:
        g.close()


def test_c1_approximation_error_scales_with_kappa_eps(orc):
    # the small workload (unit icosphere level 4, 5,120 panels) at
    # eps = 1e-6: the H-matrix solution differs from the dense LU one by
    # about kappa * eps (kappa from the oracle's exact eigenvalues); at
    # eps = 1e-12 with k_max 128 it reaches the LU solution within 1e-8
    need_gpu()
    V, T = meshgen.icosphere(4)
    A = orc.dense_matrix(V, T)
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    kappa = ev[-1] / ev[0]
    f = orc.load_vector(V, T, [3.0, 0.0, 0.0])[0]
    x_lu = orc.lu_solve(A, f)
    errs = {}
    for eps, kmax in ((1e-6, 64), (1e-12, 128)):
        g = GpuH(V, T, leaf=64, eta=1.5, eps=eps, kmax=kmax)
        try:
            x, info = g.solve(f, rel_tol=1e-13, restart=30, max_iter=5000)
            assert info.status == 0
            errs[eps] = np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu)
        finally:
            g.close()
    print("C1: kappa %.1f, |x_H - x_LU| / |x_LU| = %.2e at eps 1e-6 (kappa eps = %.1e), %.2e at eps 1e-12"
          % (kappa, errs[1e-6], kappa * 1e-6, errs[1e-12]))
    assert errs[1e-6] <= 10 * kappa * 1e-6  # the stated theory
    assert errs[1e-6] <= 20 * 1e-6  # near the measured 1.78e-6: a regression of the ACA or quadrature shows here
    assert errs[1e-12] < 1e-8
