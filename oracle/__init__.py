"""Plain FP64 CPU oracle of the H-matrix BEM hot path (arXiv 1806.11558).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_1806_11558_gb300``) never imports it, and the two share no code,
headers, tables or constant generators; the only common inputs come from
``meshgen`` (meshes and source points, no method arithmetic).

Everything here is FP64 and written to be checked by eye against the paper:

=====================  ==============================================  ========
function               paper passage                                    pinned by
=====================  ==============================================  ========
panel_geometry         Sec. 2.2 nodes X_h = panel centroids (Sec. 4.1) closed forms
morton_codes / order   Sec. 3.1 "Spatial data structure"                bit tests
cluster_tree           Sec. 2.3 (C1)-(C4), cardinality-based split      invariants
block_tree             Sec. 2.3 Algorithm 1 with Eq. 5                  invariants
entry / assemble       Sec. 2.2 Eq. 4 entries, Sec. 4.1 quadrature      see below
load_vector            Sec. 2.2 right-hand side f_i                     sphere
potential              Sec. 2.1 Eq. 2, Sec. 4.3 eps(h)                  sphere
aca_blocks             Sec. 2.3 ACA (partial pivoting)                  brute force
HMatrix.matvec         Sec. 2.3 H-matrix-vector product                 dense
gmres                  Sec. 4.1 Krylov solve (GMRES(30) reading)        LU
=====================  ==============================================  ========

Entries are pinned by: exactness of the 7-point rule on monomials of degree
<= 5; exact tiling of That x That by the Sauter-Schwab regions (polynomial
integrands); self-convergence of the singular rule; an independent
closed-form / double-exponential evaluation of touching-pair integrals; and the
unit-sphere identities S1 = 1 and S Y_lm = Y_lm / (2l+1).  No oracle function
is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from .quadrature import gauss_legendre01, tri7

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

DEFAULT_SS_ORDER = 8


def build(force: bool = False) -> str:
    """Compile hm_oracle.c into oracle/_build/liboracle.so (gcc, FP contraction off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            D = ctypes.c_double
            lib.orc_entry.restype = D
            lib.orc_entry.argtypes = [P, P, I64, I64, P, P, I, P, P]
            lib.orc_touch.restype = I
            lib.orc_touch.argtypes = [P, I64, I64]
            lib.orc_ss_points.restype = None
            lib.orc_ss_points.argtypes = [I, I64, P, P, P, P, P, P, P]
            lib.orc_assemble.restype = None
            lib.orc_assemble.argtypes = [P, P, I64, P, I64, P, P, P, I, P, P, P]
            lib.orc_load_vector.restype = None
            lib.orc_load_vector.argtypes = [P, P, I64, P, P, I64, P, P]
            lib.orc_potential.restype = None
            lib.orc_potential.argtypes = [P, P, I64, P, P, P, I64, P, P]
            lib.orc_potential_matrix.restype = None
            lib.orc_potential_matrix.argtypes = [P, P, I64, P, P, I64, P, P]
            lib.orc_admissible.restype = I
            lib.orc_admissible.argtypes = [P, P, P, P, D]
            lib.orc_block_tree.restype = I
            lib.orc_block_tree.argtypes = [I64, P, I64, D, I64, P, P, P, P]
            lib.orc_aca_blocks.restype = None
            lib.orc_aca_blocks.argtypes = [P, P, P, P, P, I, P, P, I64, P, D, I, P, P, P]
            lib.orc_aca_matrix.restype = I
            lib.orc_aca_matrix.argtypes = [I64, I64, P, D, I, P, P, P, P]
            lib.orc_hmatvec.restype = None
            lib.orc_hmatvec.argtypes = [I, I64, I64, P, P, P, I64, P, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


class Quad:
    """The quadrature data both kinds of entries use: the 7-point triangle rule
    and ``ss_order``-point Gauss-Legendre for the three regularised
    variables of the touching-pair integrals."""

    def __init__(self, ss_order: int = DEFAULT_SS_ORDER):
        self.bary, self.w7 = tri7()
        self.ss_order = int(ss_order)
        self.xgl, self.wgl = gauss_legendre01(self.ss_order)
        self.bary = _f64(self.bary)
        self.w7 = _f64(self.w7)
        self.xgl = _f64(self.xgl)
        self.wgl = _f64(self.wgl)

    def args(self):
        return (_p(self.bary), _p(self.w7), self.ss_order, _p(self.xgl), _p(self.wgl))


# --------------------------------------------------------------------------
# panels, Morton order, cluster tree, block tree
# --------------------------------------------------------------------------

def panel_geometry(V, T):
    """Centroids c_i = ((v0 + v1) + v2) / 3 (the nodes X_h, one per P0 basis
    function) and areas |T_i|, in original panel order."""
    V = _f64(V)
    T = _i32(T)
    v0, v1, v2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cent = ((v0 + v1) + v2) / 3.0
    area = 0.5 * np.linalg.norm(np.cross(v1 - v0, v2 - v0), axis=1)
    return cent, area


MORTON_BITS = 21


def morton_quantise(cent):
    """Integer grid coordinates of the centroids: lo = componentwise min,
    ext = the largest side of the bounding box (one cube for all axes),
    s = 2**21 / ext, q = min(2**21 - 1, floor((c - lo) * s))."""
    cent = _f64(cent)
    if cent.shape[0] == 0:
        return np.zeros((0, 3), dtype=np.uint64)
    lo = cent.min(axis=0)
    hi = cent.max(axis=0)
    ext = float(np.max(hi - lo))
    s = float(2 ** MORTON_BITS) / ext if ext > 0.0 else 0.0
    t = (cent - lo) * s
    q = np.floor(t).astype(np.uint64)
    return np.minimum(q, np.uint64(2 ** MORTON_BITS - 1))


def morton_interleave(q):
    """Bit b of q_x -> bit 3b+2, of q_y -> 3b+1, of q_z -> 3b."""
    q = np.asarray(q, dtype=np.uint64)
    code = np.zeros(q.shape[0], dtype=np.uint64)
    one = np.uint64(1)
    for b in range(MORTON_BITS):
        bb = np.uint64(b)
        code |= ((q[:, 0] >> bb) & one) << np.uint64(3 * b + 2)
        code |= ((q[:, 1] >> bb) & one) << np.uint64(3 * b + 1)
        code |= ((q[:, 2] >> bb) & one) << np.uint64(3 * b)
    return code


def morton_codes(cent):
    return morton_interleave(morton_quantise(cent))


def morton_order(codes):
    """perm[k] = original index of the panel at Morton position k: ascending
    by (code, original index)."""
    codes = np.asarray(codes, dtype=np.uint64)
    idx = np.arange(codes.shape[0], dtype=np.int64)
    return np.lexsort((idx, codes)).astype(np.int32)


def cluster_tree(n: int, leaf: int):
    """All clusters of the cardinality-based cluster tree as (begin, end,
    depth), children of [b, e) being [b, b + (e-b)//2) and [b + (e-b)//2, e);
    a cluster is a leaf iff its size is <= leaf (conditions (C1)-(C4))."""
    out = []
    stack = [(0, n, 0)] if n > 0 else []
    while stack:
        b, e, d = stack.pop()
        out.append((b, e, d))
        if e - b > leaf:
            m = b + (e - b) // 2
            stack.append((m, e, d + 1))
            stack.append((b, m, d + 1))
    out.sort()
    return out


def admissible(box_t, box_s, eta):
    """Eq. 5 in the squared form min(diam^2) <= eta^2 dist^2 (boxes as (lo, hi))."""
    lt, ht = (_f64(a) for a in box_t)
    ls, hs = (_f64(a) for a in box_s)
    return bool(_L().orc_admissible(_p(lt), _p(ht), _p(ls), _p(hs), float(eta) * float(eta)))


def block_tree(cent_sorted, leaf: int, eta: float):
    """Algorithm 1 from I x I.  Returns (dense, adm): int64 [n, 4] arrays of
    (row_begin, row_end, col_begin, col_end) in Morton positions, sorted by
    (row_begin, col_begin)."""
    c = _f64(cent_sorted)
    n = c.shape[0]
    cap = max(1024, 64 * n)
    while True:
        dense = np.zeros((cap, 4), dtype=np.int64)
        adm = np.zeros((cap, 4), dtype=np.int64)
        nd = ctypes.c_int64(0)
        na = ctypes.c_int64(0)
        rc = _L().orc_block_tree(n, _p(c), int(leaf), float(eta), cap, _p(dense), ctypes.byref(nd),
                                 _p(adm), ctypes.byref(na))
        if rc == 0:
            break
        cap *= 4
    dense = dense[:nd.value]
    adm = adm[:na.value]
    dense = dense[np.lexsort((dense[:, 2], dense[:, 0]))]
    adm = adm[np.lexsort((adm[:, 2], adm[:, 0]))]
    return dense, adm


class Tree:
    """Morton order + cluster tree + block tree of a mesh (Sec. 3.1, Alg. 1)."""

    def __init__(self, V, T, leaf: int = 64, eta: float = 1.5):
        self.V = _f64(V)
        self.T = _i32(T)
        self.n = self.T.shape[0]
        self.leaf = int(leaf)
        self.eta = float(eta)
        self.cent, self.area = panel_geometry(self.V, self.T)
        self.codes = morton_codes(self.cent)
        self.perm = morton_order(self.codes)
        self.iperm = np.empty_like(self.perm)
        self.iperm[self.perm] = np.arange(self.n, dtype=np.int32)
        self.cent_sorted = self.cent[self.perm]
        self.dense, self.adm = block_tree(self.cent_sorted, self.leaf, self.eta)


# --------------------------------------------------------------------------
# Galerkin entries, load vector, potential
# --------------------------------------------------------------------------

def entry(V, T, i, j, quad: Quad | None = None):
    """a_ij of Eq. 4 for original panel indices i, j."""
    quad = quad or Quad()
    V = _f64(V)
    T = _i32(T)
    return _L().orc_entry(_p(V), _p(T), int(i), int(j), *quad.args())


def touch(T, i, j):
    T = _i32(T)
    return _L().orc_touch(_p(T), int(i), int(j))


def assemble(V, T, rows, cols, quad: Quad | None = None):
    """Dense sub-matrix [a_{rows[a], cols[b]}] (original indices)."""
    quad = quad or Quad()
    V = _f64(V)
    T = _i32(T)
    rows = _i64(rows)
    cols = _i64(cols)
    out = np.empty((rows.shape[0], cols.shape[0]), dtype=np.float64)
    _L().orc_assemble(_p(V), _p(T), rows.shape[0], _p(rows), cols.shape[0], _p(cols), *quad.args(), _p(out))
    return out


def dense_matrix(V, T, quad: Quad | None = None):
    n = np.asarray(T).shape[0]
    idx = np.arange(n, dtype=np.int64)
    return assemble(V, T, idx, idx, quad)


def potential_matrix(V, T, pts, quad: Quad | None = None):
    """E with (S~ u_h)(p_k) = sum_j E[k, j] alpha_j (Sec. 2.1, single-layer
    potential ansatz), 7-point rule on every panel; [n_points, n]."""
    quad = quad or Quad()
    V = _f64(V)
    T = _i32(T)
    pts = _f64(np.asarray(pts).reshape(-1, 3))
    E = np.empty((pts.shape[0], T.shape[0]))
    _L().orc_potential_matrix(_p(V), _p(T), T.shape[0], _p(quad.bary), _p(quad.w7), pts.shape[0], _p(pts), _p(E))
    return E


def ss_points(kind: int, xi, e1, e2, e3):
    """Sauter-Schwab region maps (kind 3 = identical, 2 = common edge,
    1 = common vertex) at the given points: u, v [R, npts, 2], jac [R, npts]."""
    xi, e1, e2, e3 = (_f64(a).ravel() for a in (xi, e1, e2, e3))
    npts = xi.shape[0]
    nr = {3: 6, 2: 5, 1: 2}[kind]
    u = np.empty((nr, npts, 2))
    v = np.empty((nr, npts, 2))
    jac = np.empty((nr, npts))
    _L().orc_ss_points(int(kind), npts, _p(xi), _p(e1), _p(e2), _p(e3), _p(u), _p(v), _p(jac))
    return u, v, jac


def load_vector(V, T, sources, quad: Quad | None = None):
    """f[s, i] = int_Ti g_s dsigma with g_s(x) = 1/(4 pi |x - p_s|), 7-point rule."""
    quad = quad or Quad()
    V = _f64(V)
    T = _i32(T)
    src = _f64(np.asarray(sources).reshape(-1, 3))
    f = np.empty((src.shape[0], T.shape[0]))
    _L().orc_load_vector(_p(V), _p(T), T.shape[0], _p(quad.bary), _p(quad.w7), src.shape[0], _p(src), _p(f))
    return f


def potential(V, T, alpha, pts, quad: Quad | None = None):
    """(S~ u_h)(x) of Eq. 2 for u_h = sum_j alpha_j phi_j, at points off the surface."""
    quad = quad or Quad()
    V = _f64(V)
    T = _i32(T)
    alpha = _f64(alpha)
    pts = _f64(np.asarray(pts).reshape(-1, 3))
    out = np.empty(pts.shape[0])
    _L().orc_potential(_p(V), _p(T), T.shape[0], _p(alpha), _p(quad.bary), _p(quad.w7), pts.shape[0], _p(pts),
                       _p(out))
    return out


# --------------------------------------------------------------------------
# ACA and the H-matrix
# --------------------------------------------------------------------------

def aca_blocks(V, T, perm, blocks, eps: float, kmax: int, quad: Quad | None = None):
    """ACA with partial pivoting of each block (Morton positions).  Returns a
    list of (U [m, k], W [n, k]) with block ~ U W^T."""
    quad = quad or Quad()
    V = _f64(V)
    T = _i32(T)
    perm = _i32(perm)
    blocks = _i64(np.asarray(blocks).reshape(-1, 4))
    m = blocks[:, 1] - blocks[:, 0]
    n = blocks[:, 3] - blocks[:, 2]
    sz = (m + n) * int(kmax)
    off = np.zeros(blocks.shape[0], dtype=np.int64)
    if blocks.shape[0] > 1:
        off[1:] = np.cumsum(sz)[:-1]
    UW = np.zeros(int(sz.sum()) if blocks.shape[0] else 0)
    rank = np.zeros(blocks.shape[0], dtype=np.int32)
    if blocks.shape[0]:
        _L().orc_aca_blocks(_p(V), _p(T), _p(perm), *quad.args(), blocks.shape[0], _p(blocks), float(eps),
                            int(kmax), _p(off), _p(UW), _p(rank))
    out = []
    for b in range(blocks.shape[0]):
        k = int(rank[b])
        U = UW[off[b]:off[b] + m[b] * kmax].reshape(kmax, m[b])[:k].T.copy()
        W = UW[off[b] + m[b] * kmax:off[b] + (m[b] + n[b]) * kmax].reshape(kmax, n[b])[:k].T.copy()
        out.append((U, W))
    return out


def aca_matrix(B, eps: float, kmax: int):
    """ACA with partial pivoting of an explicit matrix B (same algorithm as
    aca_blocks).  Returns (U [m, k], W [n, k], pivot_rows, pivot_cols)."""
    B = _f64(B)
    m, n = B.shape
    kmax = int(kmax)
    U = np.zeros(m * kmax)
    W = np.zeros(n * kmax)
    pr = np.full(kmax, -1, dtype=np.int32)
    pc = np.full(kmax, -1, dtype=np.int32)
    k = _L().orc_aca_matrix(m, n, _p(B), float(eps), kmax, _p(U), _p(W), _p(pr), _p(pc))
    return (U.reshape(kmax, m)[:k].T.copy(), W.reshape(kmax, n)[:k].T.copy(), pr[:k].copy(), pc[:k].copy())


def hmatvec_raw(n, dense, dense_off, dense_val, adm, rank, uoff, woff, uw, x, trans: bool = False):
    """Apply an H-matrix given as plain arrays (Morton positions): dense block b
    row-major at dense_val[dense_off[b]:], U_b col-major (ld m) at uw[uoff[b]:],
    W_b col-major (ld n) at uw[woff[b]:], rank[b] columns."""
    dense = _i64(dense).reshape(-1, 4)
    adm = _i64(adm).reshape(-1, 4)
    y = np.empty(n)
    x = _f64(x)
    _L().orc_hmatvec(int(bool(trans)), int(n), dense.shape[0], _p(dense), _p(_i64(dense_off)), _p(_f64(dense_val)),
                     adm.shape[0], _p(adm), _p(_i32(rank)), _p(_i64(uoff)), _p(_i64(woff)), _p(_f64(uw)), _p(x),
                     _p(y))
    return y


class HMatrix:
    """FP64 CPU H-matrix: Tree + dense near field + ACA far field (Sec. 2.3, 3.3)."""

    def __init__(self, V, T, leaf=64, eta=1.5, eps=1e-6, kmax=64, quad: Quad | None = None):
        self.quad = quad or Quad()
        self.tree = Tree(V, T, leaf, eta)
        tr = self.tree
        self.n = tr.n
        # dense leaves, row-major per block
        sizes = (tr.dense[:, 1] - tr.dense[:, 0]) * (tr.dense[:, 3] - tr.dense[:, 2])
        self.dense_off = np.zeros(len(sizes), dtype=np.int64)
        if len(sizes) > 1:
            self.dense_off[1:] = np.cumsum(sizes)[:-1]
        self.dense_val = np.empty(int(sizes.sum()))
        for b, (rb, re, cb, ce) in enumerate(tr.dense):
            blk = assemble(tr.V, tr.T, tr.perm[rb:re], tr.perm[cb:ce], self.quad)
            self.dense_val[self.dense_off[b]:self.dense_off[b] + sizes[b]] = blk.ravel()
        # low-rank leaves
        fac = aca_blocks(tr.V, tr.T, tr.perm, tr.adm, eps, kmax, self.quad)
        self.rank = np.array([U.shape[1] for U, _ in fac], dtype=np.int32)
        parts, self.uoff, self.woff, o = [], [], [], 0
        for U, W in fac:
            self.uoff.append(o)
            parts.append(U.T.ravel())
            o += U.size
            self.woff.append(o)
            parts.append(W.T.ravel())
            o += W.size
        self.uoff = np.array(self.uoff, dtype=np.int64)
        self.woff = np.array(self.woff, dtype=np.int64)
        self.uw = np.concatenate(parts) if parts else np.zeros(0)

    def matvec_sorted(self, xm, trans=False):
        tr = self.tree
        return hmatvec_raw(self.n, tr.dense, self.dense_off, self.dense_val, tr.adm, self.rank, self.uoff,
                           self.woff, self.uw, xm, trans)

    def matvec(self, x, trans=False):
        """y = H x in original panel order."""
        tr = self.tree
        ym = self.matvec_sorted(np.asarray(x, dtype=np.float64)[tr.perm], trans)
        y = np.empty(self.n)
        y[tr.perm] = ym
        return y

    def stored_entries(self):
        return int(self.dense_val.size + self.uw.size)


# --------------------------------------------------------------------------
# solvers
# --------------------------------------------------------------------------

def gmres(matvec, b, restart: int = 30, tol: float = 1e-10, maxiter: int = 100000, x0=None):
    """Restarted GMRES in FP64: Arnoldi with classical Gram-Schmidt applied
    twice, Givens rotations on the Hessenberg matrix, x0 = 0 by default.  The
    Givens residual estimate ends a cycle; the true residual b - A x then
    decides convergence.  Returns (x, iterations, relative residual)."""
    b = _f64(b)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), 0, 0.0
    r = b - matvec(x)
    beta = np.linalg.norm(r)
    it = 0
    while beta > tol * bnorm and it < maxiter:
        Vb = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        Vb[0] = r / beta
        k = 0
        for j in range(restart):
            w = matvec(Vb[j])
            h = Vb[:j + 1] @ w
            w = w - Vb[:j + 1].T @ h
            h2 = Vb[:j + 1] @ w
            w = w - Vb[:j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / rho
            sn[j] = H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if abs(g[j + 1]) <= tol * bnorm or hn == 0.0 or it >= maxiter:
                break
            Vb[j + 1] = w / hn
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Vb[:k].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
    return x, it, beta / bnorm


def lu_solve(A, b):
    """Dense FP64 LU solve (LAPACK through SciPy)."""
    import scipy.linalg
    return scipy.linalg.lu_solve(scipy.linalg.lu_factor(A), b)


# --------------------------------------------------------------------------
# closed forms on the unit sphere
# --------------------------------------------------------------------------

def point_source_density(x, p):
    """Exact density u on the unit sphere with S u = 1/(4 pi |x - p|) on |x| = 1
    for an exterior source |p| > 1: with t = 1/|p| and cos(gamma) = x.p/|p|,
    u = (1 - t^2) / (4 pi |p| (1 - 2 t cos(gamma) + t^2)^(3/2))."""
    x = _f64(np.asarray(x).reshape(-1, 3))
    p = _f64(p)
    pn = np.linalg.norm(p)
    t = 1.0 / pn
    xn = x / np.linalg.norm(x, axis=1)[:, None]
    cg = xn @ (p / pn)
    return (1.0 - t * t) / (4.0 * math.pi * pn * (1.0 - 2.0 * t * cg + t * t) ** 1.5)


def point_source_potential(x, p):
    """U(x) = 1/(4 pi |x - p|), the exact interior solution."""
    x = _f64(np.asarray(x).reshape(-1, 3))
    return 1.0 / (4.0 * math.pi * np.linalg.norm(x - _f64(p)[None, :], axis=1))


# --------------------------------------------------------------------------
# Differentiation of a potential misfit through the solve (adjoint method)
# --------------------------------------------------------------------------
def misfit_loss_and_gradients(A, E, f, c, target):
    """Dense FP64 statement of the differentiated problem.

    The density alpha solves A diag(c) alpha = f (per-panel scaling c of the
    density, c = 1 at the base point), the potential at the evaluation points
    is Phi = E alpha, and the loss is L = mean_k (Phi_k - target_k)^2.  With
    g = dL/dalpha = (2/K) E^T (Phi - target), the adjoint lam solves
    (A diag(c))^T lam = g, and
        dL/df = lam,      dL/dc_j = -alpha_j (A^T lam)_j.
    Returns (L, alpha, dL/df, dL/dc).  Solves by LAPACK LU."""
    A = _f64(A)
    E = _f64(E)
    f = _f64(f)
    c = _f64(c)
    target = _f64(target)
    Ac = A * c[None, :]
    alpha = lu_solve(Ac, f)
    r = E @ alpha - target
    L = float(np.mean(r * r))
    g = (2.0 / r.shape[0]) * (E.T @ r)
    lam = lu_solve(Ac.T.copy(), g)
    return L, alpha, lam, -alpha * (A.T @ lam)
