"""Batched geometries (hm_build_forest): every geometry of the forest must
match the same mesh built on its own — the integer stage bit for bit against
the oracle, the products against the standalone GPU operator, and the
batched solve (one GMRES per geometry and right-hand side) against
standalone solves."""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu, split_dense_rows, as_set

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def forest(orc):
    torch = need_gpu()
    import paper_1806_11558_gb300 as hm
    cfg = meshgen.config("batching4")
    V, T, off = cfg["V"], cfg["T"], cfg["tri_offsets"]
    Vd, Td = torch.from_numpy(V).cuda(), torch.from_numpy(T).cuda()
    tree = hm.hm_build_forest(Vd, Td, off.tolist(), eta=1.5, leaf_size=64)
    A = hm.hm_assemble(tree, aca_eps=1e-6, aca_kmax=64, ss_order=8, factor_dtype=2, dense_dtype=1)
    yield dict(hm=hm, torch=torch, cfg=cfg, tree=tree, A=A)
    hm.hm_free(A)
    hm.hm_free(tree)


def _geom(cfg, g):
    off = cfg["tri_offsets"]
    T = cfg["T"][off[g]:off[g + 1]]
    used = np.unique(T)
    remap = np.full(cfg["V"].shape[0], -1, dtype=np.int64)
    remap[used] = np.arange(used.size)
    return np.ascontiguousarray(cfg["V"][used]), np.ascontiguousarray(remap[T].astype(np.int32))


def test_forest_tree_matches_each_geometry(orc, forest):
    hm, cfg = forest["hm"], forest["cfg"]
    n = cfg["T"].shape[0]
    info = hm.hm_tree_get_info(forest["tree"])
    assert info["n_geom"] == 4 and info["n"] == n
    perm = hm.hm_tree_get_perm(forest["tree"], n).cpu().numpy()
    dense = hm.hm_tree_get_leaves(forest["tree"], True).cpu().numpy().astype(np.int64)
    adm = hm.hm_tree_get_leaves(forest["tree"], False).cpu().numpy().astype(np.int64)
    off = cfg["tri_offsets"]
    for g in range(4):
        V, T = _geom(cfg, g)
        tr = orc.Tree(V, T, 64, 1.5)
        o = off[g]
        assert np.array_equal(perm[o:off[g + 1]] - o, tr.perm)
        in_g = lambda L: L[(L[:, 0] >= o) & (L[:, 0] < off[g + 1])] - o
        assert as_set(in_g(adm)) == as_set(tr.adm)
        assert as_set(in_g(dense)) == as_set(split_dense_rows(tr.dense, 64))
    # no block couples two geometries
    gid = np.searchsorted(off, np.arange(n), side="right") - 1
    for L in (dense, adm):
        assert np.all(gid[L[:, 0]] == gid[L[:, 2]])


def test_forest_products_and_load_vectors(orc, forest):
    hm, torch, cfg = forest["hm"], forest["torch"], forest["cfg"]
    n = cfg["T"].shape[0]
    off = cfg["tri_offsets"]
    src = torch.from_numpy(np.ascontiguousarray(cfg["sources"])).cuda()
    F = torch.empty((4, n), dtype=torch.float64, device="cuda")
    hm.hm_load_vector_geom(forest["tree"], src, F)
    x = np.random.default_rng(4).standard_normal(n)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    hm.hm_matvec(forest["A"], xd, y, prec=0)
    torch.cuda.synchronize()
    y, F = y.cpu().numpy(), F.cpu().numpy()
    for g in range(4):
        V, T = _geom(cfg, g)
        sl = slice(off[g], off[g + 1])
        fo = orc.load_vector(V, T, cfg["sources"][g])
        assert np.abs(F[:, sl] - fo).max() <= 1e-14 * np.abs(fo).max()
        alone = GpuH(V, T, leaf=64, eta=1.5, eps=1e-6, factor_dtype=2, dense_dtype=1)
        try:
            ya = alone.matvec(x[sl])
            # the same blocks, but each assembly tunes its own worker split:
            # a block that one ACA runs on a CTA worker (double-float
            # residuals) and the other on a warp worker (FP64 residuals) gets
            # factors that differ by rounding, ~1e-14 relative
            assert np.linalg.norm(y[sl] - ya) <= 1e-12 * np.linalg.norm(ya)
        finally:
            alone.close()


def test_forest_batched_solve(forest):
    hm, torch, cfg = forest["hm"], forest["torch"], forest["cfg"]
    n = cfg["T"].shape[0]
    off = cfg["tri_offsets"]
    src = torch.from_numpy(np.ascontiguousarray(cfg["sources"])).cuda()
    F = torch.empty((4, n), dtype=torch.float64, device="cuda")
    hm.hm_load_vector_geom(forest["tree"], src, F)
    X = torch.zeros_like(F)
    info = hm.hm_solve(forest["A"], F, X, rel_tol=1e-10, restart=60, precond=1, batched=1, refine=1,
                       inner_dtype=2, inner_tol=1e-2, max_refine=60, max_iter=5000)
    assert info.status == 0 and info.rel_resid <= 1e-10
    X, Fh = X.cpu().numpy(), F.cpu().numpy()
    for g in range(4):
        V, T = _geom(cfg, g)
        sl = slice(off[g], off[g + 1])
        alone = GpuH(V, T, leaf=64, eta=1.5, eps=1e-6, factor_dtype=2, dense_dtype=1)
        try:
            for r in (0, 3):
                xa, ia = alone.solve(Fh[r, sl], rel_tol=1e-10, restart=60, precond=1)
                assert np.linalg.norm(X[r, sl] - xa) <= 1e-7 * np.linalg.norm(xa)
                res = Fh[r, sl] - alone.matvec(X[r, sl])
                assert np.linalg.norm(res) <= 1.01e-10 * np.linalg.norm(Fh[r, sl])
        finally:
            alone.close()


def test_forest_with_tiny_geometries(orc):
    # geometries of 1, 2 and 37 panels beside a full icosphere: degenerate
    # trees (one-panel clusters, admissible diagonal blocks) inside one
    # forest; products against the dense oracle per geometry, and the batched
    # preconditioned, refined, graph-driven solve against it too
    torch = need_gpu()
    import paper_1806_11558_gb300 as hm
    Vi, Ti = meshgen.icosphere(2)
    parts = [
        (np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]]), np.array([[0, 1, 2]], dtype=np.int32)),
        (np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0.3]]), np.array([[0, 1, 2], [2, 1, 3]], dtype=np.int32)),
        (Vi, np.ascontiguousarray(Ti[:37])),
        (Vi * 1.3, Ti),
    ]
    Vs, Ts, off, nv = [], [], [0], 0
    for V, T in parts:
        Vs.append(V)
        Ts.append(T + nv)
        nv += V.shape[0]
        off.append(off[-1] + T.shape[0])
    V, T = np.concatenate(Vs), np.ascontiguousarray(np.concatenate(Ts).astype(np.int32))
    n = T.shape[0]
    Vd, Td = torch.from_numpy(V).cuda(), torch.from_numpy(T).cuda()
    tree = hm.hm_build_forest(Vd, Td, off, eta=1.5, leaf_size=4)
    A = hm.hm_assemble(tree, aca_eps=1e-10, aca_kmax=64, ss_order=8, factor_dtype=1, dense_dtype=1)
    try:
        rng = np.random.default_rng(8)
        x = rng.standard_normal(n)
        xd = torch.from_numpy(x).cuda()
        y = torch.empty_like(xd)
        hm.hm_matvec(A, xd, y, prec=0)
        torch.cuda.synchronize()
        y = y.cpu().numpy()
        dens = []
        for g, (Vg, Tg) in enumerate(parts):
            Ag = orc.dense_matrix(Vg, Tg)
            dens.append(Ag)
            sl = slice(off[g], off[g + 1])
            assert np.linalg.norm(y[sl] - Ag @ x[sl]) <= 1e-8 * np.linalg.norm(Ag @ x[sl])
        # two right-hand sides: systems of every geometry in lockstep
        X = np.stack([x, np.ones(n)])
        B = np.zeros_like(X)
        for g in range(len(parts)):
            sl = slice(off[g], off[g + 1])
            for r in range(2):
                B[r, sl] = dens[g] @ X[r, sl]
        Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        Xd = torch.zeros_like(Bd)
        info = hm.hm_solve(A, Bd, Xd, rel_tol=1e-12, restart=40, max_iter=3000, precond=1, batched=1, refine=1,
                           inner_dtype=1, inner_tol=1e-4, max_refine=40, use_graph=1)
        torch.cuda.synchronize()
        assert info.status == 0
        Xs = Xd.cpu().numpy()
        for r in range(2):
            assert np.linalg.norm(Xs[r] - X[r]) <= 1e-7 * np.linalg.norm(X[r])
    finally:
        hm.hm_free(A)
        hm.hm_free(tree)
