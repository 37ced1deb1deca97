"""Python binding of the GB300 H-matrix BEM library (libhm.so, C ABI in include/hm.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  The functions carry the names of the C entry points and take
CUDA tensors (torch) for the device pointers; the stream is torch's current
stream unless one is given.  There is no CPU fallback: using the binding
without a built libhm.so raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhm.so")

HM_OK, HM_EINVAL, HM_ENOMEM, HM_ECUDA, HM_ENOCONV, HM_ETIMEOUT, HM_EINTERNAL = range(7)
HM_F64, HM_F32, HM_BF16 = 0, 1, 2
STATUS_NAMES = {0: "HM_OK", 1: "HM_EINVAL", 2: "HM_ENOMEM", 3: "HM_ECUDA", 4: "HM_ENOCONV", 5: "HM_ETIMEOUT",
                6: "HM_EINTERNAL"}

EXPORTED = ["hm_build_tree", "hm_assemble", "hm_load_vector", "hm_matvec", "hm_solve", "hm_free",
            "hm_tree_get_info", "hm_tree_get_perm", "hm_tree_get_leaves", "hm_matrix_get_info",
            "hm_matrix_export", "hm_last_error", "hm_kernel_launches", "hm_matvec_noalloc", "hm_matrix_get_block",
            "hm_trace_enable", "hm_trace_read", "hm_potential", "hm_matvec_block", "hm_build_forest",
            "hm_load_vector_geom", "hm_trim", "hm_matrix_add_copy", "hm_measure_fma_peak",
            "hm_solve_scaled", "hm_matvec_scaled", "hm_set_wait_limit", "hm_set_fault_injection"]


class HMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class TreeParams(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("leaf_size", ctypes.c_int32)]


class AssembleParams(ctypes.Structure):
    _fields_ = [("aca_eps", ctypes.c_double), ("aca_kmax", ctypes.c_int32), ("ss_order", ctypes.c_int32),
                ("factor_dtype", ctypes.c_int), ("dense_dtype", ctypes.c_int), ("nearfield_fp64", ctypes.c_int32),
                ("mrhs_tcgen05", ctypes.c_int32), ("factor_tail_bits", ctypes.c_int32)]


class SolveParams(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("rel_tol", ctypes.c_double),
                ("refine", ctypes.c_int32), ("max_refine", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("inner_dtype", ctypes.c_int), ("precond", ctypes.c_int32), ("batched", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("stall_ratio", ctypes.c_double), ("resid_df", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("refine_steps", ctypes.c_int32), ("rel_resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("inner_dtype", ctypes.c_int32), ("kappa_est", ctypes.c_double)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_clusters", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("max_leaf", ctypes.c_int32), ("n_dense", ctypes.c_int64), ("n_adm", ctypes.c_int64),
                ("dense_entries", ctypes.c_int64), ("adm_rows_cols", ctypes.c_int64),
                ("n_singular", ctypes.c_int64), ("seconds", ctypes.c_double), ("n_geom", ctypes.c_int32)]


class MatrixInfo(ctypes.Structure):
    _fields_ = [("dense_entries", ctypes.c_int64), ("lr_entries", ctypes.c_int64), ("max_rank", ctypes.c_int32),
                ("kmax_hit", ctypes.c_int32), ("mean_rank", ctypes.c_double), ("s_nearfield", ctypes.c_double),
                ("s_singular", ctypes.c_double), ("s_aca", ctypes.c_double), ("s_total", ctypes.c_double),
                ("bytes_f64", ctypes.c_int64), ("bytes_low", ctypes.c_int64), ("aca_entries", ctypes.c_int64),
                ("u_entries", ctypes.c_int64), ("aca_small_sum", ctypes.c_int32), ("aca_threads", ctypes.c_int32),
                ("aca_ctas_per_sm", ctypes.c_int32), ("factor_tail_terms", ctypes.c_int64),
                ("u_tail_entries", ctypes.c_int64), ("lr_tail_entries", ctypes.c_int64)]


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


def struct_dict(s):
    return {k: getattr(s, k) for k, _ in s._fields_}


_lib = None


def lib():
    """The loaded libhm.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhm.so is not built (run __graft_entry__.build() or "
                               "python paper_1806_11558_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, D, I = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        sig = {
            "hm_build_tree": [P, I64, P, I64, P, P, P],
            "hm_assemble": [P, P, P, P],
            "hm_load_vector": [P, P, I32, P, P],
            "hm_matvec": [P, I32, I32, I, P, P, D, D, P],
            "hm_matvec_noalloc": [P, I32, I32, I, P, P, D, D, P],
            "hm_matvec_block": [P, I32, I, P, P, D, D, P],
            "hm_build_forest": [P, I64, P, I64, P, I32, P, P, P],
            "hm_load_vector_geom": [P, P, I32, P, P],
            "hm_solve": [P, I32, I32, P, P, P, P, P],
            "hm_tree_get_info": [P, P],
            "hm_tree_get_perm": [P, P],
            "hm_tree_get_leaves": [P, I32, P, I64, P],
            "hm_matrix_get_info": [P, P],
            "hm_matrix_export": [P, P, P, P, P, P, P, P, P],
            "hm_matrix_get_block": [P, I32, I64, P, P],
            "hm_trace_enable": [I32],
            "hm_potential": [P, P, I64, I32, P, P, P],
            "hm_trace_read": [P, I32, P],
            "hm_measure_fma_peak": [I, P, P],
            "hm_solve_scaled": [P, I32, I32, P, P, P, P, P, P],
            "hm_matvec_scaled": [P, I32, I32, I, P, P, P, P, D, D, P],
            "hm_set_wait_limit": [I64],
            "hm_set_fault_injection": [I64],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = I
        L.hm_free.argtypes = [P]
        L.hm_free.restype = None
        L.hm_trim.argtypes = []
        L.hm_trim.restype = None
        L.hm_matrix_add_copy.argtypes = [P, ctypes.c_int, P]
        L.hm_matrix_add_copy.restype = ctypes.c_int
        L.hm_kernel_launches.argtypes = []
        L.hm_kernel_launches.restype = ctypes.c_int64
        L.hm_last_error.argtypes = []
        L.hm_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def hm_last_error() -> str:
    return lib().hm_last_error().decode()


def hm_kernel_launches() -> int:
    return int(lib().hm_kernel_launches())


def hm_set_wait_limit(cycles: int = -1):
    """Limit (SM clock cycles) of the library's bounded device waits; < 0 restores the default."""
    _check(lib().hm_set_wait_limit(int(cycles)))


def hm_set_fault_injection(n: int = 0):
    """Fail the n-th device allocation of the library from now on (HM_ENOMEM); 0 disarms."""
    _check(lib().hm_set_fault_injection(int(n)))


def hm_measure_fma_peak(kind=HM_F64, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (HM_F64 or HM_F32)."""
    out = ctypes.c_double(0.0)
    _check(lib().hm_measure_fma_peak(int(kind), ctypes.byref(out), _stream(stream)))
    return out.value


def hm_trace_enable(on: bool = True):
    """Start (clearing it) or stop the per-kernel CUDA-event trace."""
    _check(lib().hm_trace_enable(int(bool(on))))


def hm_trace_read() -> dict:
    """{kernel name: (launches, device ms)} of the trace."""
    cnt = ctypes.c_int32(0)
    _check(lib().hm_trace_read(None, 0, ctypes.byref(cnt)))
    buf = (TraceEntry * max(1, cnt.value))()
    _check(lib().hm_trace_read(buf, cnt.value, ctypes.byref(cnt)))
    return {buf[k].name.decode(): (int(buf[k].launches), float(buf[k].ms)) for k in range(cnt.value)}


def _check(status):
    if status != HM_OK:
        raise HMError(status, hm_last_error())
    return status


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None):
    import torch
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def hm_build_tree(vertices, tris, eta=1.5, leaf_size=64, stream=None):
    """vertices: CUDA float64 [nv, 3]; tris: CUDA int32 [n, 3].  Returns a tree handle."""
    import torch
    out = ctypes.c_void_p()
    prm = TreeParams(float(eta), int(leaf_size))
    _check(lib().hm_build_tree(_ptr(vertices, torch.float64), vertices.shape[0], _ptr(tris, torch.int32),
                               tris.shape[0], ctypes.byref(prm), _stream(stream), ctypes.byref(out)))
    return out


def hm_build_forest(vertices, tris, tri_offsets, eta=1.5, leaf_size=64, stream=None):
    """Trees of several geometries in one structure: geometry g = triangles
    [tri_offsets[g], tri_offsets[g + 1]) (a host sequence of n_geom + 1 ints)."""
    import torch
    out = ctypes.c_void_p()
    prm = TreeParams(float(eta), int(leaf_size))
    off = (ctypes.c_int64 * len(tri_offsets))(*[int(v) for v in tri_offsets])
    _check(lib().hm_build_forest(_ptr(vertices, torch.float64), vertices.shape[0], _ptr(tris, torch.int32),
                                 tris.shape[0], off, len(tri_offsets) - 1, ctypes.byref(prm), _stream(stream),
                                 ctypes.byref(out)))
    return out


def hm_load_vector_geom(tree, sources, f, stream=None):
    """sources: CUDA float64 [n_geom, n_per_geom, 3]; f: [n_per_geom, n]."""
    import torch
    _check(lib().hm_load_vector_geom(tree, _ptr(sources, torch.float64), int(sources.shape[1]),
                                     _ptr(f, torch.float64), _stream(stream)))
    return f


def hm_assemble(tree, aca_eps=1e-6, aca_kmax=64, ss_order=8, factor_dtype=HM_F64, dense_dtype=HM_F64,
                nearfield_fp64=0, mrhs_tcgen05=0, factor_tail_bits=0, stream=None):
    out = ctypes.c_void_p()
    prm = AssembleParams(float(aca_eps), int(aca_kmax), int(ss_order), int(factor_dtype), int(dense_dtype),
                         int(nearfield_fp64), int(mrhs_tcgen05), int(factor_tail_bits))
    _check(lib().hm_assemble(tree, ctypes.byref(prm), _stream(stream), ctypes.byref(out)))
    return out


def hm_load_vector(tree, sources, f, stream=None):
    """sources: CUDA float64 [ns, 3]; f: CUDA float64 [ns, n] (written)."""
    import torch
    _check(lib().hm_load_vector(tree, _ptr(sources, torch.float64), sources.shape[0], _ptr(f, torch.float64),
                                _stream(stream)))
    return f


def hm_potential(tree, points, values, out=None, trans=0, stream=None):
    """Single-layer potential at points off the surface (trans = 0: [n]
    density -> [n_points] values; trans = 1: the adjoint, [n_points] -> [n])."""
    import torch
    npts = points.shape[0]
    if out is None:
        m = hm_tree_get_info(tree)["n"] if trans else npts
        out = torch.empty(m, dtype=torch.float64, device=points.device)
    _check(lib().hm_potential(tree, _ptr(points, torch.float64), int(npts), int(trans),
                              _ptr(values, torch.float64), _ptr(out, torch.float64), _stream(stream)))
    return out


def hm_matvec(A, x, y, trans=0, prec=HM_F64, alpha=1.0, beta=0.0, stream=None):
    """y = alpha op(H) x + beta y; x, y CUDA float64 [n] or [nrhs, n]."""
    import torch
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    _check(lib().hm_matvec(A, int(trans), nrhs, int(prec), _ptr(x, torch.float64), _ptr(y, torch.float64),
                           float(alpha), float(beta), _stream(stream)))
    return y


def hm_matvec_block(A, x, y, prec=HM_BF16, alpha=1.0, beta=0.0, stream=None):
    """Product for [nrhs, n] right-hand sides, 16 at a time: on the tensor
    cores with the FP32 / BF16 copies (~1e-5 relative accuracy, BF16 operand
    pairs), or (prec = HM_F64) the FP64 master in double-float arithmetic
    (~1e-14 of |H||x|)."""
    import torch
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    _check(lib().hm_matvec_block(A, nrhs, int(prec), _ptr(x, torch.float64), _ptr(y, torch.float64), float(alpha),
                                 float(beta), _stream(stream)))
    return y


def hm_matvec_noalloc(A, x, y, trans=0, prec=HM_F64, alpha=1.0, beta=0.0, stream=None):
    """hm_matvec without device allocation (working vectors in the library's
    fixed 16 MiB per-device array; see include/hm.h for the size limit and
    the rule that overlapping calls race).  Does not synchronise."""
    import torch
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    _check(lib().hm_matvec_noalloc(A, int(trans), nrhs, int(prec), _ptr(x, torch.float64), _ptr(y, torch.float64),
                                   float(alpha), float(beta), _stream(stream)))
    return y


def hm_solve(A, b, x, trans=0, restart=30, max_iter=3000, rel_tol=1e-10, refine=0, max_refine=20, inner_tol=1e-4,
             inner_dtype=HM_F32, precond=0, batched=0, use_graph=0, stall_ratio=0.5, resid_df=0, stream=None,
             raise_on_noconv=True):
    """Solves op(H) x = b; returns the SolveInfo of the (last) right-hand side."""
    import torch
    nrhs = 1 if b.dim() == 1 else b.shape[0]
    prm = SolveParams(int(restart), int(max_iter), float(rel_tol), int(refine), int(max_refine), float(inner_tol),
                      int(inner_dtype), int(precond), int(batched), int(use_graph), float(stall_ratio),
                      int(resid_df))
    info = SolveInfo()
    st = lib().hm_solve(A, int(trans), nrhs, _ptr(b, torch.float64), _ptr(x, torch.float64), ctypes.byref(prm),
                        _stream(stream), ctypes.byref(info))
    if st == HM_ENOCONV and not raise_on_noconv:
        return info
    _check(st)
    return info


def hm_solve_scaled(A, b, c, x, trans=0, restart=30, max_iter=3000, rel_tol=1e-10, refine=0, max_refine=20,
                    inner_tol=1e-4, inner_dtype=HM_F32, precond=0, batched=0, use_graph=0, stall_ratio=0.5,
                    resid_df=0, stream=None, raise_on_noconv=True):
    """Solves op(H diag(c)) x = b (c: CUDA float64 [n]); returns the SolveInfo."""
    import torch
    nrhs = 1 if b.dim() == 1 else b.shape[0]
    prm = SolveParams(int(restart), int(max_iter), float(rel_tol), int(refine), int(max_refine), float(inner_tol),
                      int(inner_dtype), int(precond), int(batched), int(use_graph), float(stall_ratio),
                      int(resid_df))
    info = SolveInfo()
    st = lib().hm_solve_scaled(A, int(trans), nrhs, _ptr(c, torch.float64), _ptr(b, torch.float64),
                               _ptr(x, torch.float64), ctypes.byref(prm), _stream(stream), ctypes.byref(info))
    if st == HM_ENOCONV and not raise_on_noconv:
        return info
    _check(st)
    return info


def hm_matvec_scaled(A, x, y, trans=0, prec=HM_F64, left=None, right=None, alpha=1.0, beta=0.0, stream=None):
    """y = alpha diag(left) op(H) diag(right) x + beta y (left / right: CUDA float64 [n] or None)."""
    import torch
    nrhs = 1 if x.dim() == 1 else x.shape[0]
    _check(lib().hm_matvec_scaled(A, int(trans), nrhs, int(prec), _ptr(left, torch.float64),
                                  _ptr(right, torch.float64), _ptr(x, torch.float64), _ptr(y, torch.float64),
                                  float(alpha), float(beta), _stream(stream)))
    return y


def hm_matrix_add_copy(A, dtype, stream=None):
    """Adds the FP32 (HM_F32) or BF16 (HM_BF16) copy to an assembled matrix."""
    _check(lib().hm_matrix_add_copy(A, int(dtype), _stream(stream)))


def hm_trim():
    """Returns the device blocks the library keeps for reuse to the driver."""
    lib().hm_trim()


def hm_free(handle):
    if handle:
        lib().hm_free(handle)


def hm_tree_get_info(tree) -> dict:
    info = TreeInfo()
    _check(lib().hm_tree_get_info(tree, ctypes.byref(info)))
    return struct_dict(info)


def hm_tree_get_perm(tree, n):
    import torch
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(lib().hm_tree_get_perm(tree, _ptr(perm)))
    return perm


def hm_tree_get_leaves(tree, dense: bool):
    import torch
    cnt = ctypes.c_int64(0)
    _check(lib().hm_tree_get_leaves(tree, int(dense), None, 0, ctypes.byref(cnt)))
    out = torch.empty((max(cnt.value, 1), 4), dtype=torch.int32, device="cuda")
    _check(lib().hm_tree_get_leaves(tree, int(dense), _ptr(out), cnt.value, ctypes.byref(cnt)))
    return out[:cnt.value]


def hm_matrix_get_info(A) -> dict:
    info = MatrixInfo()
    _check(lib().hm_matrix_get_info(A, ctypes.byref(info)))
    return struct_dict(info)


def hm_matrix_get_block(A, dense: bool, index: int, m: int, n: int, stream=None):
    """Leaf `index` of the H-matrix as a dense (m, n) CUDA float64 tensor."""
    import torch
    out = torch.empty((m, n), dtype=torch.float64, device="cuda")
    _check(lib().hm_matrix_get_block(A, int(dense), int(index), _ptr(out), _stream(stream)))
    return out


def hm_matrix_export(A, n_dense: int, n_adm: int):
    """Host copy of the FP64 H-matrix (numpy arrays, plain layout of hm.h)."""
    import numpy as np
    nd = ctypes.c_int64(0)
    nl = ctypes.c_int64(0)
    _check(lib().hm_matrix_export(A, None, None, None, None, None, None, ctypes.byref(nd), ctypes.byref(nl)))
    dense = np.zeros(max(nd.value, 1))
    doff = np.zeros(max(n_dense, 1), dtype=np.int64)
    rank = np.zeros(max(n_adm, 1), dtype=np.int32)
    uw = np.zeros(max(nl.value, 1))
    uoff = np.zeros(max(n_adm, 1), dtype=np.int64)
    woff = np.zeros(max(n_adm, 1), dtype=np.int64)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(lib().hm_matrix_export(A, P(dense), P(doff), P(rank), P(uw), P(uoff), P(woff), ctypes.byref(nd),
                                  ctypes.byref(nl)))
    return dict(dense=dense[:nd.value], dense_off=doff[:n_dense], rank=rank[:n_adm], uw=uw[:nl.value],
                u_off=uoff[:n_adm], w_off=woff[:n_adm])
