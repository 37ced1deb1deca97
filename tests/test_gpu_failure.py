"""Failure paths on the GPU, made without a GPU fault.

* The bounded wait of the near-field assembly (TMA-staged panel tiles) with
  its limit set to 0 cycles gives up before polling: the assembly returns
  HM_ETIMEOUT, after the blocks have waited (with the default limit) for the
  copies they started, and the context stays usable: the next assembly with
  the default limit gives the same operator as before.
* The same for the tcgen05 / TMEM row pass of the 16-right-hand-side product
  (bulk copies, cp.async gathers and MMAs in flight when the waits give up):
  the product returns HM_ETIMEOUT, every role drains what it started, the
  TMEM is freed, and the next product is the same bit for bit.
* Injected allocation failures (hm_set_fault_injection) at every position of
  a build + assembly + product: each failing call returns HM_ENOMEM, frees
  what it had allocated (device memory back to its level before the call
  once the library's block cache is trimmed), and the operator built
  afterwards is the same bit for bit.
"""
import numpy as np
import pytest

import meshgen

from hm_gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _build(hm, torch, Vd, Td, x):
    tree = hm.hm_build_tree(Vd, Td, eta=1.5, leaf_size=64)
    A = None
    try:
        A = hm.hm_assemble(tree, aca_eps=1e-6, factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32)
        y = torch.empty_like(x)
        hm.hm_matvec(A, x, y)
        torch.cuda.synchronize()
        return y
    finally:
        if A is not None:
            hm.hm_free(A)
        hm.hm_free(tree)


@pytest.fixture(scope="module")
def mesh():
    torch = need_gpu()
    import paper_1806_11558_gb300 as hm
    V, T = meshgen.icosphere(3)
    Vd, Td = torch.from_numpy(V).cuda(), torch.from_numpy(T).cuda()
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(T.shape[0])).cuda()
    y0 = _build(hm, torch, Vd, Td, x)
    return hm, torch, Vd, Td, x, y0


def test_wait_limit_zero_times_out_and_context_survives(mesh):
    hm, torch, Vd, Td, x, y0 = mesh
    tree = hm.hm_build_tree(Vd, Td, eta=1.5, leaf_size=64)
    try:
        hm.hm_set_wait_limit(0)
        with pytest.raises(hm.HMError) as e:
            hm.hm_assemble(tree, aca_eps=1e-6, factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32)
        assert e.value.status == hm.HM_ETIMEOUT
        assert "timed out" in str(e.value)
    finally:
        hm.hm_set_wait_limit(-1)
        hm.hm_free(tree)
    torch.cuda.synchronize()  # the context still answers
    assert torch.equal(_build(hm, torch, Vd, Td, x), y0)


def test_wait_limit_zero_in_the_tensor_memory_row_pass(mesh):
    hm, torch, Vd, Td, x, y0 = mesh
    tree = hm.hm_build_tree(Vd, Td, eta=1.5, leaf_size=64)
    A = hm.hm_assemble(tree, aca_eps=1e-6, factor_dtype=hm.HM_F32, dense_dtype=hm.HM_F32, mrhs_tcgen05=1)
    try:
        X = torch.from_numpy(np.random.default_rng(5).standard_normal((16, x.numel()))).cuda()
        Y0, Y = torch.empty_like(X), torch.empty_like(X)
        hm.hm_matvec_block(A, X, Y0, prec=hm.HM_F32)
        torch.cuda.synchronize()
        try:
            hm.hm_set_wait_limit(0)
            with pytest.raises(hm.HMError) as e:
                hm.hm_matvec_block(A, X, Y, prec=hm.HM_F32)
            assert e.value.status == hm.HM_ETIMEOUT
            assert "row pass gave up" in str(e.value)
        finally:
            hm.hm_set_wait_limit(-1)
        torch.cuda.synchronize()  # the context still answers
        for _ in range(2):
            hm.hm_matvec_block(A, X, Y, prec=hm.HM_F32)
            torch.cuda.synchronize()
            assert torch.equal(Y, Y0)
    finally:
        hm.hm_free(A)
        hm.hm_free(tree)


def test_injected_allocation_failures_free_everything(mesh):
    hm, torch, Vd, Td, x, y0 = mesh
    hm.hm_trim()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = []
    k = 1
    while True:
        hm.hm_set_fault_injection(k)
        try:
            y = _build(hm, torch, Vd, Td, x)
        except hm.HMError as e:
            assert e.status == hm.HM_ENOMEM, e
            assert "injected allocation failure" in str(e)
            failed.append(k)
        else:
            assert torch.equal(y, y0)
            break  # k is past the last allocation: the whole sequence ran
        finally:
            hm.hm_set_fault_injection(0)
        hm.hm_trim()
        torch.cuda.synchronize()
        free = torch.cuda.mem_get_info()[0]
        assert free >= free0 - (4 << 20), (k, free0 - free)
        k += 1
        assert k < 5000, "more allocations than expected"
    assert len(failed) >= 20 and failed == list(range(1, k))
    assert torch.equal(_build(hm, torch, Vd, Td, x), y0)
