"""The allocation-free H-matrix-vector product (hm_matvec_noalloc).

It exists for callers that may not allocate device memory while it runs (a
fixed memory budget or pool of their own, where a cudaMalloc / cudaFree would
fail or disturb their accounting).  It must give the same result as
hm_matvec, call after call, and must not change the device's free memory.
This file is collected last, so a run that stops at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import GpuH, need_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_matvec_matches_hm_matvec_on_consecutive_calls():
    torch = need_gpu()
    import paper_1806_11558_gb300 as hm
    V, T = meshgen.icosphere(3)
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32)
    try:
        rng = np.random.default_rng(11)
        xs = [torch.from_numpy(rng.standard_normal(g.n)).cuda() for _ in range(2)]
        for prec in (hm.HM_F64, hm.HM_F32):
            refs = []
            for x in xs:
                y = torch.empty_like(x)
                hm.hm_matvec(g.A, x, y, prec=prec)
                refs.append(y)
            outs = [torch.full_like(x, float("nan")) for x in xs]  # allocated before the calls
            torch.cuda.synchronize()
            # two calls in a row sharing the scratch array; the first call on a
            # device also looks up the array's address (and may load the module)
            hm.hm_matvec_noalloc(g.A, xs[0], outs[0], prec=prec)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            hm.hm_matvec_noalloc(g.A, xs[1], outs[1], prec=prec)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
            for y, r in zip(outs, refs):
                err = float(torch.linalg.norm(y - r) / torch.linalg.norm(r))
                assert err <= 1e-12, (prec, err)
    finally:
        g.close()


def test_noalloc_matvec_rejects_what_it_cannot_do():
    """trans = 1 is not offered, and a problem whose working vectors exceed the
    fixed array (2,097,152 doubles; a level-6 icosphere needs more) is refused
    with the required size in the message, before any device work."""
    torch = need_gpu()
    import paper_1806_11558_gb300 as hm
    V, T = meshgen.icosphere(3)
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-8, factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32)
    try:
        x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        with pytest.raises(hm.HMError) as e:
            hm.hm_matvec_noalloc(g.A, x, torch.empty_like(x), trans=1)
        assert e.value.status == hm.HM_EINVAL and "trans" in str(e.value)
    finally:
        g.close()
    V, T = meshgen.icosphere(6)
    g = GpuH(V, T, leaf=64, eta=1.5, eps=1e-4)
    try:
        x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        y = torch.full_like(x, 7.0)
        with pytest.raises(hm.HMError) as e:
            hm.hm_matvec_noalloc(g.A, x, y)
        assert e.value.status == hm.HM_EINVAL
        assert "needs" in str(e.value) and "2097152" in str(e.value)
        torch.cuda.synchronize()
        assert float(y.min()) == 7.0 and float(y.max()) == 7.0  # nothing was written
    finally:
        g.close()
