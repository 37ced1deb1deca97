"""Batched lockstep GMRES (hm_solve with batched = 1) against one solve per
right-hand side on the same operator; the refined form runs its inner
solves through the 16-right-hand-side tensor-core product."""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sphere(orc):
    need_gpu()
    V, T, _ = meshgen.bump_sphere(4, 1808)
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=2, dense_dtype=1)
    yield g
    g.close()


def _rhs(g, nrhs):
    return g.load_vector(meshgen.point_sources(77, nrhs))


def _solve(g, B, **kw):
    torch = g.torch
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    Xd = torch.zeros_like(Bd)
    info = g.hm.hm_solve(g.A, Bd, Xd, **kw)
    torch.cuda.synchronize()
    return Xd.cpu().numpy(), info


@pytest.mark.parametrize("precond", [0, 1])
def test_batched_fp64_matches_single_solves(sphere, precond):
    g = sphere
    B = _rhs(g, 5)
    X, info = _solve(g, B, rel_tol=1e-12, restart=40, precond=precond, batched=1, max_iter=2000)
    assert info.status == 0 and info.rel_resid <= 1e-12
    for r in range(B.shape[0]):
        xr, ir = g.solve(B[r], rel_tol=1e-12, restart=40, precond=precond)
        assert np.linalg.norm(X[r] - xr) <= 1e-9 * np.linalg.norm(xr)
        res = B[r] - g.matvec(X[r])
        assert np.linalg.norm(res) <= 1.01e-12 * np.linalg.norm(B[r])


@pytest.mark.parametrize("nrhs", [16, 20])
def test_batched_refined_matches_fp64(sphere, nrhs):
    g = sphere
    B = _rhs(g, nrhs)
    X, info = _solve(g, B, rel_tol=1e-12, restart=60, precond=1, batched=1, refine=1, inner_dtype=2,
                     inner_tol=1e-2, max_refine=60, max_iter=5000)
    assert info.status == 0 and info.rel_resid <= 1e-12 and info.refine_steps >= 1
    for r in (0, nrhs // 2, nrhs - 1):
        xr, ir = g.solve(B[r], rel_tol=1e-12, restart=60, precond=1)
        assert np.linalg.norm(X[r] - xr) <= 1e-8 * np.linalg.norm(xr)
        res = B[r] - g.matvec(X[r])
        assert np.linalg.norm(res) <= 1.01e-12 * np.linalg.norm(B[r])


def test_batched_zero_rhs_column(sphere):
    g = sphere
    B = _rhs(g, 3)
    B[1] = 0.0
    X, info = _solve(g, B, rel_tol=1e-12, restart=40, precond=1, batched=1, refine=1, inner_dtype=2,
                     inner_tol=1e-2, max_refine=60, max_iter=5000)
    assert info.status == 0
    assert np.all(X[1] == 0.0)


def _oracle_solutions(orc, g, B, tol):
    """oracle.gmres on the exported FP64 operator, one system at a time."""
    perm = g.perm()
    ex = g.export()
    dl, al = g.leaves(True), g.leaves(False)

    def mv(x):
        ym = orc.hmatvec_raw(g.n, dl, ex["dense_off"], ex["dense"], al, ex["rank"], ex["u_off"], ex["w_off"],
                             ex["uw"], x[perm])
        y = np.empty(g.n)
        y[perm] = ym
        return y

    return np.array([orc.gmres(mv, B[r], restart=60, tol=tol, maxiter=20000)[0] for r in range(B.shape[0])])


@pytest.mark.parametrize("form", ["fp64", "refined_bf16", "refined_f32", "refined_f32_df"])
def test_batched_solutions_match_the_oracle_gmres(orc, sphere, form):
    g = sphere
    B = _rhs(g, 17)  # one full pass of 16 right-hand sides and a ragged one
    kw = dict(rel_tol=1e-12, restart=60, precond=1, batched=1, max_iter=5000)
    if form != "fp64":
        kw.update(refine=1, inner_dtype=2 if form == "refined_bf16" else 1,
                  inner_tol=1e-2 if form == "refined_bf16" else 1e-4, max_refine=60)
        if form.startswith("refined_f32"):
            g.hm.hm_matrix_add_copy(g.A, 1)
        if form == "refined_f32_df":
            kw.update(resid_df=1)  # outer residuals by the double-float 16-column product
    X, info = _solve(g, B, **kw)
    assert info.status == 0 and info.rel_resid <= 1e-12
    Xo = _oracle_solutions(orc, g, B, 1e-12)
    err = np.linalg.norm(X - Xo, axis=1) / np.linalg.norm(Xo, axis=1)
    assert err.max() <= 1e-8, err
    if form == "refined_f32_df":
        # the FP64 residual of the solutions, by the oracle: the double-float
        # residual the solver stopped on is within ~1e-14 of |H||x| of it
        perm = g.perm()
        ex = g.export()
        dl, al = g.leaves(True), g.leaves(False)
        for r in range(B.shape[0]):
            hx = np.empty(g.n)
            hx[perm] = orc.hmatvec_raw(g.n, dl, ex["dense_off"], ex["dense"], al, ex["rank"], ex["u_off"],
                                       ex["w_off"], ex["uw"], X[r][perm])
            assert np.linalg.norm(B[r] - hx) <= 1.05e-12 * np.linalg.norm(B[r]), r
