"""The library's device block cache: freed buffers of 1 MiB or more are kept
for later allocations instead of being unmapped.  A cached block holds the
previous owner's data, so an assembly that reuses blocks must still build
the same operator bit for bit (nothing may depend on fresh memory), and
hm_trim must hand the blocks back to the driver."""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu

pytestmark = pytest.mark.gpu


def _products(g, xs, hm):
    torch = g.torch
    out = []
    for prec in (hm.HM_F64, hm.HM_F32):
        for x in xs:
            y = torch.empty_like(x)
            hm.hm_matvec(g.A, x, y, prec=prec)
            out.append(y.cpu().numpy())
    torch.cuda.synchronize()
    return out


def test_reassembly_on_cached_blocks_is_identical(orc):
    torch = need_gpu()
    import paper_1806_11558_gb300 as hm
    V, T, _ = meshgen.bump_sphere(4, 1814)
    rng = np.random.default_rng(5)
    xs = [torch.from_numpy(rng.standard_normal(T.shape[0])).cuda() for _ in range(2)]
    b = None
    runs = []
    for rep in range(3):
        # rep 0 on fresh memory (after a trim), reps 1 and 2 on the blocks
        # the previous assembly and solve released
        if rep == 0:
            hm.hm_trim()
        g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32)
        try:
            if b is None:
                b = g.load_vector(meshgen.point_sources(61, 1))[0]
            ys = _products(g, xs, hm)
            x64, i64 = g.solve(b, rel_tol=1e-12, restart=40, precond=1)
            xm, im = g.solve(b, rel_tol=1e-12, restart=40, precond=1, refine=1, inner_dtype=hm.HM_F32,
                             inner_tol=1e-4, max_refine=40, max_iter=5000)
            runs.append((ys, x64, i64.iters, xm, im.iters))
        finally:
            g.close()
    for ys, x64, it64, xm, itm in runs[1:]:
        for a, c in zip(runs[0][0], ys):
            assert np.array_equal(a, c)
        assert np.array_equal(runs[0][1], x64) and runs[0][2] == it64
        assert np.array_equal(runs[0][3], xm) and runs[0][4] == itm


def test_trim_returns_memory(orc):
    torch = need_gpu()
    import paper_1806_11558_gb300 as hm
    V, T, _ = meshgen.bump_sphere(4, 1815)
    hm.hm_trim()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32)
    g.close()
    torch.cuda.synchronize()
    free_cached = torch.cuda.mem_get_info()[0]
    hm.hm_trim()
    free1 = torch.cuda.mem_get_info()[0]
    # the freed matrix stays cached until the trim, which returns it
    assert free1 >= free_cached
    assert abs(free1 - free0) <= 64 << 20


@pytest.mark.parametrize("dtype", [1, 2])
def test_add_copy_matches_assembled_copy(orc, dtype):
    # a copy added after the assembly is the same rounding of the same FP64
    # master as the copy the assembly keeps: products agree bit for bit
    torch = need_gpu()
    import paper_1806_11558_gb300 as hm
    V, T, _ = meshgen.bump_sphere(4, 1816)
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=dtype, dense_dtype=hm.HM_F32)
    try:
        A2 = hm.hm_assemble(g.tree, aca_eps=1e-8, aca_kmax=64, ss_order=8)
        try:
            with pytest.raises(hm.HMError):
                hm.hm_matvec(A2, torch.zeros(g.n, dtype=torch.float64, device="cuda"),
                             torch.zeros(g.n, dtype=torch.float64, device="cuda"), prec=dtype)
            hm.hm_matrix_add_copy(A2, dtype)
            hm.hm_matrix_add_copy(A2, dtype)  # a second call keeps the copy
            x = torch.from_numpy(np.random.default_rng(6).standard_normal(g.n)).cuda()
            y1, y2 = torch.empty_like(x), torch.empty_like(x)
            hm.hm_matvec(g.A, x, y1, prec=dtype)
            hm.hm_matvec(A2, x, y2, prec=dtype)
            torch.cuda.synchronize()
            assert torch.equal(y1, y2)
        finally:
            hm.hm_free(A2)
    finally:
        g.close()
