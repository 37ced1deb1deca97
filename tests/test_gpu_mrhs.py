"""Tensor-core product with many right-hand sides (hm_matvec_block) against
the one-right-hand-side product of the same low-precision copy: the BF16
operand pairs keep ~16 significant bits, so the two agree to ~1e-5."""
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


@pytest.mark.parametrize("name,mesh,leaf", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [1, 2], ids=["f32", "bf16"])
def test_block_product_matches_single_products(name, mesh, leaf, prec):
    torch = need_gpu()
    V, T = mesh()
    g = GpuH(V, T, leaf=leaf, eta=1.5, eps=1e-6, factor_dtype=prec, dense_dtype=1)
    try:
        hm = g.hm
        rng = np.random.default_rng(9)
        for nrhs in (16, 5, 20):
            X = rng.standard_normal((nrhs, g.n))
            Xd = torch.from_numpy(X).cuda()
            Y = torch.empty_like(Xd)
            hm.hm_matvec_block(g.A, Xd, Y, prec=prec)
            ref = torch.empty_like(Xd)
            for r in range(nrhs):
                hm.hm_matvec(g.A, Xd[r].contiguous(), ref[r], prec=prec)
            torch.cuda.synchronize()
            err = torch.linalg.norm(Y - ref, dim=1) / torch.linalg.norm(ref, dim=1)
            assert float(err.max()) <= 5e-5, (nrhs, err.max().item())
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


def test_block_product_rejects_fp64():
    torch = need_gpu()
    V, T = meshgen.icosphere(2)
    g = GpuH(V, T, eps=1e-6, factor_dtype=1, dense_dtype=1)
    try:
        x = torch.zeros((2, g.n), dtype=torch.float64, device="cuda")
        with pytest.raises(g.hm.HMError):
            g.hm.hm_matvec_block(g.A, x, x.clone(), prec=0)
    finally:
        g.close()
