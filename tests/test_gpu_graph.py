"""The CUDA-graph form of GMRES (hm_solve with use_graph = 1: the Arnoldi
steps of a cycle as one WHILE conditional node, the stop decided on the
device) against the host-driven loop.  Both launch the same kernels with the
same arguments in the same order, and every reduction has a fixed order, so
the iterates, the step counts and the solutions agree bit for bit."""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sphere(orc):
    need_gpu()
    V, T, _ = meshgen.bump_sphere(4, 1811)
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=2, dense_dtype=1)
    yield g
    g.close()


@pytest.fixture(scope="module")
def sphere32(orc):
    need_gpu()
    V, T, _ = meshgen.bump_sphere(4, 1812)
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=1, dense_dtype=1)
    yield g
    g.close()


def _pair(g, B, **kw):
    torch = g.torch
    out = []
    for use_graph in (0, 1):
        Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        Xd = torch.zeros_like(Bd)
        info = g.hm.hm_solve(g.A, Bd, Xd, use_graph=use_graph, raise_on_noconv=False, **kw)
        torch.cuda.synchronize()
        out.append((Xd.cpu().numpy(), info))
    (x0, i0), (x1, i1) = out
    assert (i0.status, i0.iters, i0.restarts, i0.refine_steps) == (i1.status, i1.iters, i1.restarts, i1.refine_steps)
    assert i0.rel_resid == i1.rel_resid
    assert np.array_equal(x0, x1)
    return x1, i1


@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("trans", [0, 1])
def test_graph_fp64_identical(sphere, precond, trans):
    g = sphere
    b = g.load_vector(meshgen.point_sources(91, 1))[0]
    x, info = _pair(g, b, rel_tol=1e-12, restart=30, precond=precond, trans=trans, max_iter=3000)
    assert info.status == 0 and info.rel_resid <= 1e-12 and info.restarts >= 2


@pytest.mark.parametrize("inner", [1, 2])
def test_graph_refined_identical(sphere, sphere32, inner):
    g = sphere32 if inner == 1 else sphere
    b = g.load_vector(meshgen.point_sources(92, 1))[0]
    x, info = _pair(g, b, rel_tol=1e-12, restart=40, precond=1, refine=1, inner_dtype=inner, inner_tol=1e-3,
                    max_refine=40, max_iter=5000)
    assert info.status == 0 and info.refine_steps >= 2


def test_graph_step_limit(sphere):
    # max_iter in the middle of a cycle: the device-side limit ends the loop
    # at the same step as the host loop, and the solve reports non-convergence
    g = sphere
    b = g.load_vector(meshgen.point_sources(93, 1))[0]
    x, info = _pair(g, b, rel_tol=1e-14, restart=8, precond=0, max_iter=13)
    assert info.iters == 13 and info.status != 0


@pytest.mark.parametrize("refine", [0, 1, 2], ids=["fp64", "refined", "refined_df_residuals"])
def test_graph_batched_identical(sphere, refine):
    # refined: FP32 Krylov vectors in the inner solves (6 right-hand sides);
    # refined_df_residuals: and the outer residuals by the double-float product
    g = sphere
    B = g.load_vector(meshgen.point_sources(94, 6))
    kw = dict(rel_tol=1e-12, restart=40, precond=1, batched=1, max_iter=5000)
    if refine:
        kw.update(refine=1, inner_dtype=2, inner_tol=1e-2, max_refine=60, resid_df=int(refine == 2))
    X, info = _pair(g, B, **kw)
    assert info.status == 0 and info.rel_resid <= 1e-12
    res = B[3] - g.matvec(X[3])
    assert np.linalg.norm(res) <= 1.01e-12 * np.linalg.norm(B[3])


def test_graph_batched_step_limit(sphere):
    g = sphere
    B = g.load_vector(meshgen.point_sources(95, 3))
    X, info = _pair(g, B, rel_tol=1e-14, restart=6, precond=0, batched=1, max_iter=11)
    assert info.iters == 11 and info.status != 0


def test_graph_counts_replayed_launches(sphere):
    # the launch counter covers the kernels each replay runs: a graph solve
    # reports as many launches as the host loop
    g = sphere
    hm = g.hm
    b = g.load_vector(meshgen.point_sources(96, 1))[0]
    counts = []
    for use_graph in (0, 1):
        c0 = hm.hm_kernel_launches()
        g.solve(b, rel_tol=1e-12, restart=30, precond=1, use_graph=use_graph)
        counts.append(hm.hm_kernel_launches() - c0)
    # the graph form adds one copy kernel per step and drops nothing
    assert counts[1] >= counts[0]
