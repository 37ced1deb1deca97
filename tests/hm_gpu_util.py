"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class GpuH:
    """Tree + H-matrix built through the C ABI, freed on close()."""

    def __init__(self, V, T, leaf=64, eta=1.5, eps=1e-6, kmax=64, ss_order=8, factor_dtype=0, dense_dtype=0,
                 nearfield_fp64=0, mrhs_tcgen05=0, factor_tail_bits=0):
        torch = need_gpu()
        import paper_1806_11558_gb300 as hm
        self.hm = hm
        self.torch = torch
        self.V, self.T = V, T
        self.n = T.shape[0]
        self.Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        self.Td = torch.from_numpy(np.ascontiguousarray(T)).cuda()
        self.tree = hm.hm_build_tree(self.Vd, self.Td, eta=eta, leaf_size=leaf)
        self.A = None
        if eps is not None:
            self.A = hm.hm_assemble(self.tree, aca_eps=eps, aca_kmax=kmax, ss_order=ss_order,
                                    factor_dtype=factor_dtype, dense_dtype=dense_dtype,
                                    nearfield_fp64=nearfield_fp64, mrhs_tcgen05=mrhs_tcgen05,
                                    factor_tail_bits=factor_tail_bits)

    def perm(self):
        return self.hm.hm_tree_get_perm(self.tree, self.n).cpu().numpy()

    def leaves(self, dense):
        return self.hm.hm_tree_get_leaves(self.tree, dense).cpu().numpy().astype(np.int64)

    def info(self):
        return self.hm.hm_tree_get_info(self.tree)

    def export(self):
        ti = self.info()
        return self.hm.hm_matrix_export(self.A, ti["n_dense"], ti["n_adm"])

    def block(self, dense, index, blk):
        rb, re, cb, ce = blk
        out = self.hm.hm_matrix_get_block(self.A, dense, index, int(re - rb), int(ce - cb))
        self.torch.cuda.synchronize()
        return out.cpu().numpy()

    def matvec(self, x, prec=0, trans=0):
        torch = self.torch
        xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
        yd = torch.empty_like(xd)
        self.hm.hm_matvec(self.A, xd, yd, prec=prec, trans=trans)
        torch.cuda.synchronize()
        return yd.cpu().numpy()

    def load_vector(self, sources):
        torch = self.torch
        src = torch.tensor(np.asarray(sources, dtype=np.float64).reshape(-1, 3)).cuda()
        f = torch.empty((src.shape[0], self.n), dtype=torch.float64, device="cuda")
        self.hm.hm_load_vector(self.tree, src, f)
        torch.cuda.synchronize()
        return f.cpu().numpy()

    def solve(self, b, **kw):
        torch = self.torch
        bd = torch.from_numpy(np.ascontiguousarray(b, dtype=np.float64)).cuda()
        xd = torch.zeros_like(bd)
        info = self.hm.hm_solve(self.A, bd, xd, **kw)
        torch.cuda.synchronize()
        return xd.cpu().numpy(), info

    def close(self):
        if self.A is not None:
            self.hm.hm_free(self.A)
            self.A = None
        if self.tree is not None:
            self.hm.hm_free(self.tree)
            self.tree = None


def split_dense_rows(dense, leaf):
    """Non-admissible leaves whose row cluster is not a leaf cluster are stored
    as its two children's row blocks (same entries); apply that to a list of
    leaves from Algorithm 1."""
    out = []
    for rb, re, cb, ce in np.asarray(dense, dtype=np.int64):
        if re - rb > leaf:
            m = rb + (re - rb) // 2
            out += [(rb, m, cb, ce), (m, re, cb, ce)]
        else:
            out.append((rb, re, cb, ce))
    return np.array(out, dtype=np.int64).reshape(-1, 4)


def as_set(blocks):
    return set(map(tuple, np.asarray(blocks, dtype=np.int64).reshape(-1, 4).tolist()))
