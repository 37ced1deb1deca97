"""Iterative refinement that stops contracting: an outer step whose FP64
residual is above stall_ratio times the previous one raises the inner
precision (BF16 -> FP32, making the FP32 copies from the FP64 master when
the assembly kept only BF16 factors; FP32 -> FP64).  A tiny stall_ratio
forces every step to count as a stall, which walks the whole ladder."""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu

pytestmark = pytest.mark.gpu

F64, F32, BF16 = 0, 1, 2


def _mesh():
    V, T, _ = meshgen.bump_sphere(4, 1813)
    return V, T


def test_refine_contracts_keeps_bf16(orc):
    need_gpu()
    V, T = _mesh()
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=BF16, dense_dtype=F32)
    try:
        b = g.load_vector(meshgen.point_sources(97, 1))[0]
        x, info = g.solve(b, rel_tol=1e-12, restart=40, precond=1, refine=1, inner_dtype=BF16, inner_tol=1e-3,
                          max_refine=40, max_iter=5000)
        assert info.status == 0 and info.inner_dtype == BF16 and info.refine_steps >= 2
    finally:
        g.close()


@pytest.mark.parametrize("batched", [0, 1])
def test_refine_stall_walks_to_fp64(orc, batched):
    need_gpu()
    V, T = _mesh()
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=BF16, dense_dtype=F64)
    try:
        B = g.load_vector(meshgen.point_sources(98, 3))
        torch = g.torch
        Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        Xd = torch.zeros_like(Bd)
        info = g.hm.hm_solve(g.A, Bd, Xd, rel_tol=1e-12, restart=40, precond=1, refine=1, inner_dtype=BF16,
                             inner_tol=1e-2, max_refine=60, max_iter=8000, batched=batched, stall_ratio=1e-30)
        torch.cuda.synchronize()
        X = Xd.cpu().numpy()
        assert info.status == 0 and info.inner_dtype == F64 and info.refine_steps >= 3
        # the FP32 copies made on the way are kept with the matrix: an FP32
        # inner solve is now accepted
        x32, i32 = g.solve(B[0], rel_tol=1e-12, restart=40, precond=1, refine=1, inner_dtype=F32, inner_tol=1e-4,
                           max_refine=40, max_iter=5000)
        assert i32.status == 0 and i32.inner_dtype == F32
        for r in range(B.shape[0]):
            xr, _ = g.solve(B[r], rel_tol=1e-12, restart=40, precond=1)
            assert np.linalg.norm(X[r] - xr) <= 1e-8 * np.linalg.norm(xr)
    finally:
        g.close()


def test_stall_ratio_nan_rejected(orc):
    need_gpu()
    V, T = _mesh()
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-6, factor_dtype=BF16, dense_dtype=F32)
    try:
        b = g.load_vector(meshgen.point_sources(99, 1))[0]
        with pytest.raises(g.hm.HMError):
            g.solve(b, refine=1, inner_dtype=BF16, stall_ratio=float("nan"))
    finally:
        g.close()
