// aca.cu -- batched adaptive cross approximation of all admissible blocks.
//
// Sec. 2.3: every admissible leaf tau x sigma is approximated by a rank-k
// matrix U W^T built by ACA ("a pivoted Gauss elimination ... by successive
// rank-one updates"), with matrix entries evaluated on the fly.  Sec. 3.1
// "Batching": all blocks of uneven size are handled by one launch.
//
// ACA with partial pivoting, per block (m x n, local indices):
//   i_1 = 0.  Step r: residual row  ~u = B(i_r, :) - sum_l U(i_r, l) W(:, l)^T,
//   column pivot j_r = argmax_{unused j} |~u_j| (lowest j on ties),
//   delta = ~u(j_r); a zero row (delta == 0 at r = 1, |delta| <= 2^-50 |delta_1|
//   later) is marked used and replaced by the lowest unused row;
//   W(:, r) = ~u / delta (as ~u times the reciprocal of delta),
//   U(:, r) = B(:, j_r) - sum_l W(j_r, l) U(:, l);
//   ||S_r||^2 += 2 sum_{l<r} (u_r.u_l)(w_l.w_r) + ||u_r||^2 ||w_r||^2;
//   stop when ||u_r|| ||w_r|| <= eps ||S_r|| or r = min(m, n, kmax);
//   next row i_{r+1} = argmax_{unused i} |u_r(i)|.
//
// One persistent kernel.  Each CTA first takes large blocks (m + n above a
// threshold) from a work counter, largest first, and runs the ACA with all
// its threads (CTA-wide argmax and dot products through shared memory); when
// none are left each warp takes small blocks on its own (shuffle argmax,
// shuffle dot products, no block barriers).  All reductions have a fixed
// order, so the factors are identical from run to run.  Converged factors are
// copied from per-worker scratch to a bump-allocated arena; blocks that do not
// fit are reported and re-run after the arena grows.  The CTA workers keep the
// factor columns as float pairs and form the residuals in double-float
// arithmetic; the warp workers keep them in FP64 and form the residuals with
// FP64 FMAs (measured: the float-pair residuals are 24% faster on the large
// blocks of a level-8 sphere with 80-panel leaves, 5-8% slower on the small
// blocks, where the FP32 units are already the busier pipe).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "entry.cuh"
#include "ff.cuh"

namespace hm {

// CTA sizes of the persistent kernel (the autotuner picks one; 128 by default)
constexpr int ACA_THREADS = 128;
constexpr int ACA_MAX_WARPS = 8;
constexpr int SMALL_MAX_DIM = 256;  // warp-mode blocks: m, n <= this
constexpr int HUGE_SUM = 2560;      // CTA-mode blocks with m + n above this use the large scratch
// per-warp shared doubles in warp mode: fixed record, U/W row values, bitmaps, norm terms
constexpr int WARP_SMEM_DOUBLES = 32 + MAX_KMAX + (SMALL_MAX_DIM + 31) / 32 + (2 + 2 * MAX_KMAX + 1) / 2;

struct AcaArgs {
    const double *pt;
    const float *pf;
    int64_t npad;
    const double *V;
    const int32_t *adm;
    const int32_t *work;  // blocks to approximate, largest first: [0, n_big) CTA-wide, then warp-wide
    int64_t n_big, n_work;
    double eps;
    int kmax;
    QuadParams qp;
    double *scr_big;
    int64_t big_stride;
    double *scr_small;
    int64_t small_stride;
    int big_words_r, big_words_c;  // bitmap words in CTA mode
    int big_ctas;                  // CTAs that take the huge blocks
    int64_t n_huge;                // work[0, n_huge): huge blocks (m + n > HUGE_SUM), CTA-wide, big_ctas CTAs
    double *scr_med;               // per-CTA scratch of the other CTA-wide blocks
    int64_t med_stride;
    unsigned long long *q_huge;
    double *arena;
    int64_t arena_cap;
    unsigned long long *arena_top;
    int32_t *rank;
    int64_t *uw_off;
    unsigned long long *q_big, *q_small;
    int *kmax_hit;
    const int32_t *todo;  // optional subset of block ids (re-run after overflow)
    int64_t n_todo;
};

struct Best {
    double a;  // |value|
    int idx;   // index (INT_MAX = none)
    double v;  // signed value
};

__device__ __forceinline__ bool better(const Best &x, const Best &y) {
    return x.a > y.a || (x.a == y.a && x.idx < y.idx);
}

__device__ __forceinline__ Best warp_argmax(Best b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Best c;
        c.a = __shfl_xor_sync(0xffffffffu, b.a, o);
        c.idx = __shfl_xor_sync(0xffffffffu, b.idx, o);
        c.v = __shfl_xor_sync(0xffffffffu, b.v, o);
        if (better(c, b)) b = c;
    }
    return b;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// shared scratch of one ACA worker (CTA or warp)
struct AcaShared {
    float *fix;     // [64]  fixed panel record (float panel table row)
    double *vec;    // [kmax] U(i_r, :) or W(j_r, :)
    double *red;    // [warps] sum partials (CTA mode)
    Best *bred;     // [warps] argmax partials (CTA mode)
    uint32_t *urow, *ucol;
    long long *ibc; // broadcast slot (CTA mode)
    float *stage;   // norm terms per warp: CTA [warps][NORM_STRIDE], warp [NORM_STRIDE]
    float *res;     // reduced norm terms [NORM_STRIDE]
};

constexpr int NORM_STRIDE = 2 + 2 * MAX_KMAX;

// Terms of the Frobenius norm of the approximant after step r, accumulated in
// FP32 from the high parts of the factor columns (the estimate only
// decides when to stop): res[0] = |u_r|^2, res[1] = |w_r|^2,
// res[2 + l] = u_r . u_l, res[2 + r + l] = w_l . w_r (l < r).  One pass over
// the columns, per-warp shuffle reductions, one shared-memory round.
template <bool CTA, int NT>
__device__ void norm_terms(const float *Uf, const float *Wf, int m, int n, int r, const AcaShared &sh) {
    const int gs = CTA ? NT : 32, t = CTA ? (int)threadIdx.x : (int)(threadIdx.x & 31);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nvals = 2 + 2 * r;
    const float *ur = Uf + (int64_t)r * m, *wr = Wf + (int64_t)r * n;
    float *st = CTA ? sh.stage + warp * NORM_STRIDE : sh.stage;
    for (int c0 = 0; c0 < nvals; c0 += 8) {
        float acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
        for (int k = t; k < m; k += gs) {
            const float u = ur[k];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int v = c0 + c;
                if (v == 0) acc[c] = fmaf(u, u, acc[c]);
                else if (v >= 2 && v < 2 + r) acc[c] = fmaf(u, Uf[(int64_t)(v - 2) * m + k], acc[c]);
            }
        }
        for (int j = t; j < n; j += gs) {
            const float w = wr[j];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int v = c0 + c;
                if (v == 1) acc[c] = fmaf(w, w, acc[c]);
                else if (v >= 2 + r && v < nvals) acc[c] = fmaf(w, Wf[(int64_t)(v - 2 - r) * n + j], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float a = acc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0 && c0 + c < nvals) st[c0 + c] = a;
        }
    }
    if (CTA) {
        __syncthreads();
        for (int v = t; v < nvals; v += gs) {
            float a = 0.0f;
            for (int w = 0; w < NT / 32; ++w) a += sh.stage[w * NORM_STRIDE + v];
            sh.res[v] = a;
        }
        __syncthreads();
    } else {
        __syncwarp();
    }
}

template <bool CTA, int NT>
__device__ void norm_terms(const FF *Uf, const FF *Wf, int m, int n, int r, const AcaShared &sh) {
    const int gs = CTA ? NT : 32, t = CTA ? (int)threadIdx.x : (int)(threadIdx.x & 31);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nvals = 2 + 2 * r;
    const FF *ur = Uf + (int64_t)r * m, *wr = Wf + (int64_t)r * n;
    float *st = CTA ? sh.stage + warp * NORM_STRIDE : sh.stage;
    for (int c0 = 0; c0 < nvals; c0 += 8) {
        float acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
        for (int k = t; k < m; k += gs) {
            const float u = ur[k].h;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int v = c0 + c;
                if (v == 0) acc[c] = fmaf(u, u, acc[c]);
                else if (v >= 2 && v < 2 + r) acc[c] = fmaf(u, Uf[(int64_t)(v - 2) * m + k].h, acc[c]);
            }
        }
        for (int j = t; j < n; j += gs) {
            const float w = wr[j].h;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int v = c0 + c;
                if (v == 1) acc[c] = fmaf(w, w, acc[c]);
                else if (v >= 2 + r && v < nvals) acc[c] = fmaf(w, Wf[(int64_t)(v - 2 - r) * n + j].h, acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float a = acc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0 && c0 + c < nvals) st[c0 + c] = a;
        }
    }
    if (CTA) {
        __syncthreads();
        for (int v = t; v < nvals; v += gs) {
            float a = 0.0f;
            for (int w = 0; w < NT / 32; ++w) a += sh.stage[w * NORM_STRIDE + v];
            sh.res[v] = a;
        }
        __syncthreads();
    } else {
        __syncwarp();
    }
}

template <bool CTA, int NT>
struct Grp {
    __device__ __forceinline__ static int size() { return CTA ? NT : 32; }
    __device__ __forceinline__ static int rank() { return CTA ? (int)threadIdx.x : (int)(threadIdx.x & 31); }
    __device__ __forceinline__ static void sync() {
        if (CTA) __syncthreads();
        else __syncwarp();
    }
    __device__ __forceinline__ static double sum(double v, const AcaShared &sh) {
        v = warp_sum(v);
        if (!CTA) return v;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) sh.red[w] = v;
        __syncthreads();
        double t = 0.0;
        for (int k = 0; k < NT / 32; ++k) t += sh.red[k];
        __syncthreads();
        return t;
    }
    __device__ __forceinline__ static Best argmax(Best b, const AcaShared &sh) {
        b = warp_argmax(b);
        if (!CTA) return b;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) sh.bred[w] = b;
        __syncthreads();
        Best t = sh.bred[0];
        for (int k = 1; k < NT / 32; ++k)
            if (better(sh.bred[k], t)) t = sh.bred[k];
        __syncthreads();
        return t;
    }
    // value of group thread 0, to every thread of the group
    __device__ __forceinline__ static long long bcast(long long v, const AcaShared &sh) {
        if (!CTA) return __shfl_sync(0xffffffffu, v, 0);
        if (threadIdx.x == 0) *sh.ibc = v;
        __syncthreads();
        long long r = *sh.ibc;
        __syncthreads();
        return r;
    }
};

__device__ __forceinline__ bool bit(const uint32_t *bm, int k) { return (bm[k >> 5] >> (k & 31)) & 1u; }

// One out-of-line copy of the far-field evaluation shared by every call site
// (row and column passes, CTA and warp workers).
__device__ __noinline__ static FF far_entry(const float *r, int rs, const float *c, int cs, const float *wh,
                                            const float *wl) {
    FF e;
    regular_entry_ff2(r, rs, c, cs, wh, wl, e.h, e.l);
    return e;
}

// Entry of the Galerkin matrix for the row panel at Morton position gi and the
// column panel at gj; `fix` is the shared-memory record of the panel that is
// fixed during the pass (the row panel when fixed_is_row, else the column
// panel), the other record is read from the float panel table.  Far-field
// pairs in float-float; touching pairs (which admissible blocks do not contain
// in practice) by the FP64 regularised rule.
__device__ __forceinline__ FF aca_entry(const float *fix, bool fixed_is_row, int64_t gi, int64_t gj,
                                        const AcaArgs &A) {
    const int64_t var = fixed_is_row ? gj : gi;
    const float *rec = A.pf + var;
    const int64_t st = A.npad;
    const int32_t vf[3] = {__float_as_int(fix[PF_VID]), __float_as_int(fix[PF_VID + 1]),
                           __float_as_int(fix[PF_VID + 2])};
    const int32_t vv[3] = {__float_as_int(rec[PF_VID * st]), __float_as_int(rec[(PF_VID + 1) * st]),
                           __float_as_int(rec[(PF_VID + 2) * st])};
    const int kind = shared_vertices(vf, vv);
    if (kind) {
        const double ai = A.pt[(int64_t)PT_AREA * A.npad + gi], aj = A.pt[(int64_t)PT_AREA * A.npad + gj];
        return ff_from(fixed_is_row ? singular_entry_serial(A.V, vf, vv, kind, ai, aj, A.qp)
                                    : singular_entry_serial(A.V, vv, vf, kind, ai, aj, A.qp));
    }
    // The regular rule sums over the points of the row-role panel in a rolled
    // loop that reads that panel's record as it goes, and loads the
    // column-role record into registers up front.  G(x, y) = G(y, x), so the
    // pair is evaluated with the fixed (shared-memory) record in the row role
    // in both passes: the varying record, read from L2, is then loaded once
    // per entry instead of once per outer step.  The value is the same entry
    // up to rounding (~1e-14 relative, the order of the double-float sums).
    return far_entry(fix, 1, rec, (int)st, A.qp.w_h, A.qp.w_l);
}

// ACA of one block (CTA workers); U (m x kmax) and W (n x kmax) column-major
// in scratch, as float pairs: the residual rows and columns (entry minus the
// rank-one terms so far) are formed in double-float arithmetic on the FP32
// units, to ~2^-48 of the largest term, like the entries themselves.
template <bool CTA, int NT>
__device__ int aca_block(const AcaArgs &A, int rb, int m, int cb, int n, FF *U, FF *W, const AcaShared &sh,
                         bool *hit_kmax) {
    using G = Grp<CTA, NT>;
    const int gs = G::size(), t = G::rank();
    const int wr = (m + 31) >> 5, wc = (n + 31) >> 5;
    for (int k = t; k < wr; k += gs) sh.urow[k] = 0u;
    for (int k = t; k < wc; k += gs) sh.ucol[k] = 0u;
    G::sync();
    const int rmax = min(A.kmax, min(m, n));
    const double tiny = 8.881784197001252e-16;  // 2^-50
    FF *vec = reinterpret_cast<FF *>(sh.vec);
    int r = 0, i = 0;
    double s2 = 0.0, delta1 = 0.0;
    bool converged = false;
    while (r < rmax) {
        // ---- residual of row i ----
        for (int q = t; q < PF_ROWS; q += gs) sh.fix[q] = A.pf[(int64_t)q * A.npad + rb + i];
        for (int l = t; l < r; l += gs) vec[l] = U[(int64_t)l * m + i];
        G::sync();
        Best best{-1.0, 0x7fffffff, 0.0};
        for (int j = t; j < n; j += gs) {
            const FF e = aca_entry(sh.fix, true, rb + i, cb + j, A);
            float hs = e.h, lo = e.l;
            for (int l = 0; l < r; ++l) ff_sub_prod(hs, lo, vec[l], W[(int64_t)l * n + j]);
            FF v;
            fast_two_sum(hs, lo, v.h, v.l);
            W[(int64_t)r * n + j] = v;
            if (!bit(sh.ucol, j)) {
                const double vd = ff_to(v);
                const Best c{fabs(vd), j, vd};
                if (better(c, best)) best = c;
            }
        }
        best = G::argmax(best, sh);
        if (t == 0) sh.urow[i >> 5] |= 1u << (i & 31);
        G::sync();
        const double delta = best.v;
        const bool zero_row = (r == 0) ? (delta == 0.0) : (fabs(delta) <= tiny * delta1);
        if (zero_row || best.idx == 0x7fffffff) {
            // lowest unused row
            int cand = 0x7fffffff;
            for (int k = t; k < m; k += gs)
                if (!bit(sh.urow, k)) { cand = k; break; }
            Best c{0.0, cand, 0.0};
            c = G::argmax(c, sh);
            if (c.idx == 0x7fffffff) break;
            i = c.idx;
            continue;
        }
        if (r == 0) delta1 = fabs(delta);
        const int jp = best.idx;
        const FF inv_delta = ff_from(1.0 / delta);
        for (int j = t; j < n; j += gs) W[(int64_t)r * n + j] = ff_mul(W[(int64_t)r * n + j], inv_delta);
        // ---- residual of column jp ----
        for (int q = t; q < PF_ROWS; q += gs) sh.fix[q] = A.pf[(int64_t)q * A.npad + cb + jp];
        for (int l = t; l < r; l += gs) vec[l] = W[(int64_t)l * n + jp];
        G::sync();
        Best nb{-1.0, 0x7fffffff, 0.0};
        for (int k = t; k < m; k += gs) {
            const FF e = aca_entry(sh.fix, false, rb + k, cb + jp, A);
            float hs = e.h, lo = e.l;
            for (int l = 0; l < r; ++l) ff_sub_prod(hs, lo, vec[l], U[(int64_t)l * m + k]);
            FF u;
            fast_two_sum(hs, lo, u.h, u.l);
            U[(int64_t)r * m + k] = u;
            if (!bit(sh.urow, k)) {
                const double ud = ff_to(u);
                const Best c{fabs(ud), k, ud};
                if (better(c, nb)) nb = c;
            }
        }
        if (t == 0) sh.ucol[jp >> 5] |= 1u << (jp & 31);
        // ---- Frobenius norm of the approximant ----
        norm_terms<CTA, NT>(U, W, m, n, r, sh);
        const float *res = CTA ? sh.res : sh.stage;
        const double nu2 = res[0], nw2 = res[1];
        double cross = 0.0;
        for (int l = 0; l < r; ++l) cross += (double)res[2 + l] * (double)res[2 + r + l];
        s2 = s2 + 2.0 * cross + nu2 * nw2;
        ++r;
        nb = G::argmax(nb, sh);
        if (sqrt(nu2) * sqrt(nw2) <= A.eps * sqrt(s2)) { converged = true; break; }
        if (nb.idx == 0x7fffffff) { converged = true; break; }
        i = nb.idx;
        G::sync();
    }
    *hit_kmax = !converged && r == A.kmax && r < min(m, n);
    return r;
}

// copy the first k columns of U and W to the arena (bump allocation)
template <bool CTA, int NT>
__device__ void aca_store(const AcaArgs &A, int64_t b, int m, int n, int k, const FF *U, const FF *W,
                          const AcaShared &sh) {
    using G = Grp<CTA, NT>;
    const int gs = G::size(), t = G::rank();
    const int64_t need = (int64_t)k * (m + n);
    long long off = 0;
    if (t == 0) off = (long long)atomicAdd(A.arena_top, (unsigned long long)need);
    off = G::bcast(off, sh);
    if (t == 0) A.rank[b] = k;
    if ((int64_t)off + need > A.arena_cap) {
        if (t == 0) A.uw_off[b] = -1;
        return;
    }
    if (t == 0) A.uw_off[b] = (int64_t)off;
    // U_b column-major (m x k); W_b row-major (n x k): row j of W_b holds the
    // k coefficients of column j of the block, which the projection W_b^T x
    // reads contiguously
    double *dst = A.arena + off;
    const int64_t mk = (int64_t)m * k, nk = (int64_t)n * k;
    for (int64_t e = t; e < mk; e += gs) dst[e] = ff_to(U[e]);
    for (int64_t e = t; e < nk; e += gs) {
        const int64_t j = e / k, l = e - j * k;
        dst[mk + e] = ff_to(W[l * n + j]);
    }
}

// The same ACA with the factor columns in FP64 (U, W) plus FP32 shadows (Uf,
// Wf) for the norm terms, the rank-one updates of the residuals in FP64.
// Used by the warp workers (small blocks), where the FP32 units are the
// busier pipe; the CTA workers (large blocks) use the float-pair form.
template <bool CTA, int NT>
__device__ int aca_block_d(const AcaArgs &A, int rb, int m, int cb, int n, double *U, double *W, float *Uf, float *Wf,
                         const AcaShared &sh, bool *hit_kmax) {
    using G = Grp<CTA, NT>;
    const int gs = G::size(), t = G::rank();
    const int wr = (m + 31) >> 5, wc = (n + 31) >> 5;
    for (int k = t; k < wr; k += gs) sh.urow[k] = 0u;
    for (int k = t; k < wc; k += gs) sh.ucol[k] = 0u;
    G::sync();
    const int rmax = min(A.kmax, min(m, n));
    const double tiny = 8.881784197001252e-16;  // 2^-50
    int r = 0, i = 0;
    double s2 = 0.0, delta1 = 0.0;
    bool converged = false;
    while (r < rmax) {
        // ---- residual of row i ----
        for (int q = t; q < PF_ROWS; q += gs) sh.fix[q] = A.pf[(int64_t)q * A.npad + rb + i];
        for (int l = t; l < r; l += gs) sh.vec[l] = U[(int64_t)l * m + i];
        G::sync();
        Best best{-1.0, 0x7fffffff, 0.0};
        for (int j = t; j < n; j += gs) {
            double v = ff_to(aca_entry(sh.fix, true, rb + i, cb + j, A));
            for (int l = 0; l < r; ++l) v -= sh.vec[l] * W[(int64_t)l * n + j];
            W[(int64_t)r * n + j] = v;
            if (!bit(sh.ucol, j)) {
                const Best c{fabs(v), j, v};
                if (better(c, best)) best = c;
            }
        }
        best = G::argmax(best, sh);
        if (t == 0) sh.urow[i >> 5] |= 1u << (i & 31);
        G::sync();
        const double delta = best.v;
        const bool zero_row = (r == 0) ? (delta == 0.0) : (fabs(delta) <= tiny * delta1);
        if (zero_row || best.idx == 0x7fffffff) {
            // lowest unused row
            int cand = 0x7fffffff;
            for (int k = t; k < m; k += gs)
                if (!bit(sh.urow, k)) { cand = k; break; }
            Best c{0.0, cand, 0.0};
            c = G::argmax(c, sh);
            if (c.idx == 0x7fffffff) break;
            i = c.idx;
            continue;
        }
        if (r == 0) delta1 = fabs(delta);
        const int jp = best.idx;
        const double inv_delta = 1.0 / delta;
        for (int j = t; j < n; j += gs) {
            const double w = W[(int64_t)r * n + j] * inv_delta;
            W[(int64_t)r * n + j] = w;
            Wf[(int64_t)r * n + j] = (float)w;
        }
        // ---- residual of column jp ----
        for (int q = t; q < PF_ROWS; q += gs) sh.fix[q] = A.pf[(int64_t)q * A.npad + cb + jp];
        for (int l = t; l < r; l += gs) sh.vec[l] = W[(int64_t)l * n + jp];
        G::sync();
        Best nb{-1.0, 0x7fffffff, 0.0};
        for (int k = t; k < m; k += gs) {
            double u = ff_to(aca_entry(sh.fix, false, rb + k, cb + jp, A));
            for (int l = 0; l < r; ++l) u -= sh.vec[l] * U[(int64_t)l * m + k];
            U[(int64_t)r * m + k] = u;
            Uf[(int64_t)r * m + k] = (float)u;
            if (!bit(sh.urow, k)) {
                const Best c{fabs(u), k, u};
                if (better(c, nb)) nb = c;
            }
        }
        if (t == 0) sh.ucol[jp >> 5] |= 1u << (jp & 31);
        // ---- Frobenius norm of the approximant ----
        norm_terms<CTA, NT>(Uf, Wf, m, n, r, sh);
        const float *res = CTA ? sh.res : sh.stage;
        const double nu2 = res[0], nw2 = res[1];
        double cross = 0.0;
        for (int l = 0; l < r; ++l) cross += (double)res[2 + l] * (double)res[2 + r + l];
        s2 = s2 + 2.0 * cross + nu2 * nw2;
        ++r;
        nb = G::argmax(nb, sh);
        if (sqrt(nu2) * sqrt(nw2) <= A.eps * sqrt(s2)) { converged = true; break; }
        if (nb.idx == 0x7fffffff) { converged = true; break; }
        i = nb.idx;
        G::sync();
    }
    *hit_kmax = !converged && r == A.kmax && r < min(m, n);
    return r;
}

template <bool CTA, int NT>
__device__ void aca_store(const AcaArgs &A, int64_t b, int m, int n, int k, const double *U, const double *W,
                          const AcaShared &sh) {
    using G = Grp<CTA, NT>;
    const int gs = G::size(), t = G::rank();
    const int64_t need = (int64_t)k * (m + n);
    long long off = 0;
    if (t == 0) off = (long long)atomicAdd(A.arena_top, (unsigned long long)need);
    off = G::bcast(off, sh);
    if (t == 0) A.rank[b] = k;
    if ((int64_t)off + need > A.arena_cap) {
        if (t == 0) A.uw_off[b] = -1;
        return;
    }
    if (t == 0) A.uw_off[b] = (int64_t)off;
    // U_b column-major (m x k); W_b row-major (n x k): row j of W_b holds the
    // k coefficients of column j of the block, which the projection W_b^T x
    // reads contiguously
    double *dst = A.arena + off;
    const int64_t mk = (int64_t)m * k, nk = (int64_t)n * k;
    for (int64_t e = t; e < mk; e += gs) dst[e] = U[e];
    for (int64_t e = t; e < nk; e += gs) {
        const int64_t j = e / k, l = e - j * k;
        dst[mk + e] = W[l * n + j];
    }
}

// NT threads per CTA, MINB CTAs per SM in the register budget (about 100
// registers per thread for every NT)
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) aca_kernel(AcaArgs A) {
    constexpr int WARPS = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_red[WARPS];
    __shared__ Best s_bred[WARPS];
    __shared__ long long s_ibc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // ---------------- phase 1: large blocks, whole CTA ----------------
    // 1a: the huge blocks (and an overflow re-run) on the first big_ctas CTAs,
    // whose scratch fits any block; 1b: the other large blocks on every CTA
    for (int tier = 0; tier < 2; ++tier) {
        if (tier == 0 && (int)blockIdx.x >= A.big_ctas) continue;
        if (tier == 1 && A.todo) break;
        AcaShared sh;
        double *d = reinterpret_cast<double *>(smem_raw);
        sh.fix = reinterpret_cast<float *>(d);
        sh.vec = d + 32;
        sh.red = s_red;
        sh.bred = s_bred;
        sh.ibc = &s_ibc;
        sh.urow = reinterpret_cast<uint32_t *>(d + 32 + MAX_KMAX);
        sh.ucol = sh.urow + A.big_words_r;
        sh.stage = reinterpret_cast<float *>(sh.ucol + A.big_words_c + ((A.big_words_r + A.big_words_c) & 1));
        sh.res = sh.stage + WARPS * NORM_STRIDE;
        double *U = tier == 0 ? A.scr_big + (int64_t)blockIdx.x * A.big_stride
                              : A.scr_med + (int64_t)blockIdx.x * A.med_stride;
        for (;;) {
            long long q = 0;
            if (threadIdx.x == 0) q = (long long)atomicAdd(tier == 0 ? A.q_huge : A.q_big, 1ull);
            q = Grp<true, NT>::bcast(q, sh);
            const int64_t q0 = tier == 0 ? 0 : A.n_huge;
            const int64_t qend = A.todo ? A.n_todo : (tier == 0 ? A.n_huge : A.n_big);
            if (q0 + q >= qend) break;
            const int64_t b = A.todo ? A.todo[q] : A.work[q0 + q];
            const int32_t rb = A.adm[4 * b], re = A.adm[4 * b + 1], cb = A.adm[4 * b + 2], ce = A.adm[4 * b + 3];
            const int m = re - rb, n = ce - cb;
            FF *Uff = reinterpret_cast<FF *>(U);
            FF *W = Uff + (int64_t)m * A.kmax;
            bool hit = false;
            const int k = aca_block<true, NT>(A, rb, m, cb, n, Uff, W, sh, &hit);
            if (hit && threadIdx.x == 0) atomicAdd(A.kmax_hit, 1);
            __syncthreads();
            aca_store<true, NT>(A, b, m, n, k, Uff, W, sh);
            __syncthreads();
        }
    }
    if (A.todo) return;

    // ---------------- phase 2: small blocks, one warp each ----------------
    {
        AcaShared sh;
        const int words = (SMALL_MAX_DIM + 31) / 32;
        double *d = reinterpret_cast<double *>(smem_raw) + (int64_t)warp * WARP_SMEM_DOUBLES;
        sh.fix = reinterpret_cast<float *>(d);
        sh.vec = d + 32;
        sh.red = nullptr;
        sh.bred = nullptr;
        sh.ibc = nullptr;
        sh.urow = reinterpret_cast<uint32_t *>(d + 32 + MAX_KMAX);
        sh.ucol = sh.urow + words;
        sh.stage = reinterpret_cast<float *>(d + 32 + MAX_KMAX + words);
        sh.res = sh.stage;
        double *U = A.scr_small + ((int64_t)blockIdx.x * WARPS + warp) * A.small_stride;
        for (;;) {
            int q = 0;
            if (lane == 0) q = (int)atomicAdd(A.q_small, 1ull);
            q = __shfl_sync(0xffffffffu, q, 0);
            if (A.n_big + q >= A.n_work) break;
            const int64_t b = A.work[A.n_big + q];
            const int32_t rb = A.adm[4 * b], re = A.adm[4 * b + 1], cb = A.adm[4 * b + 2], ce = A.adm[4 * b + 3];
            const int m = re - rb, n = ce - cb;
            double *W = U + (int64_t)m * A.kmax;
            float *Uf = reinterpret_cast<float *>(W + (int64_t)n * A.kmax);
            float *Wf = Uf + (int64_t)m * A.kmax;
            bool hit = false;
            const int k = aca_block_d<false, NT>(A, rb, m, cb, n, U, W, Uf, Wf, sh, &hit);
            if (hit && lane == 0) atomicAdd(A.kmax_hit, 1);
            __syncwarp();
            aca_store<false, NT>(A, b, m, n, k, U, W, sh);
            __syncwarp();
        }
    }
}

__global__ void aca_overflow_list(const int64_t *uw_off, int64_t na, int32_t *list, int *count) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x)
        if (uw_off[b] < 0) list[atomicAdd(count, 1)] = (int32_t)b;
}

// blocks below the diagonal with a partner take its rank (their factors are
// the partner's, transposed)
__global__ void mirror_rank_kernel(const int32_t *adm, const int32_t *tp, int64_t na, int32_t *rank, int64_t *uw_off) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = tp[b];
        if (p >= 0 && adm[4 * b] > adm[4 * b + 2]) {
            rank[b] = rank[p];
            uw_off[b] = uw_off[p];
        }
    }
}

// k_b (m_b + n_b) per block, or k_b m_b (rows_only)
__global__ void lr_size_kernel(const int32_t *adm, const int32_t *rank, int64_t na, int rows_only, int64_t *out) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x)
        out[b] = (int64_t)rank[b] *
                 ((adm[4 * b + 1] - adm[4 * b]) + (rows_only ? 0 : (adm[4 * b + 3] - adm[4 * b + 2])));
}

__global__ void rank_to_i64(const int32_t *rank, int64_t na, int64_t *out) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x)
        out[b] = rank[b];
}

__global__ void rank_stats(const int32_t *rank, int64_t na, unsigned long long *sum, int *maxr) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(sum, (unsigned long long)rank[b]);
        atomicMax(maxr, rank[b]);
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
// ACA of every admissible leaf.  Output: A->rank, A->t_off, A->total_rank,
// A->lr_entries, and the factors in `uw` (per block U_b column-major then W_b
// row-major at uw_off[b]), exactly sized.
// key of the factor-arena size hint: (admissible blocks, sum of m + n over
// the approximated ones, eps, kmax)
using ArenaKey = std::tuple<int64_t, int64_t, double, int>;

void assemble_aca(const hm_tree *tr, hm_matrix *A, const QuadParams &qp, cudaStream_t s, double *sec, DBuf &uw,
                  DBuf &uw_off) {
    const int64_t na = tr->n_adm;
    const int kmax = A->params.aca_kmax;
    A->rank.alloc(sizeof(int32_t) * std::max<int64_t>(na, 1));
    uw_off.alloc(sizeof(int64_t) * std::max<int64_t>(na, 1));
    A->t_off.alloc(sizeof(int64_t) * (na + 1));
    if (na == 0) {
        uw.alloc(16);
        A->lr_entries = 0;
        A->total_rank = 0;
        HM_CUDA_CHECK(cudaMemsetAsync(A->t_off.p, 0, sizeof(int64_t), s));
        *sec = 0.0;
        return;
    }
    // block sizes on the host; the matrix is symmetric, so of a pair of blocks
    // with swapped ranges only the one above the diagonal is approximated
    std::vector<int32_t> h_adm(4 * na), h_tp(na);
    HM_CUDA_CHECK(cudaMemcpyAsync(h_adm.data(), tr->adm.p, sizeof(int32_t) * 4 * na, cudaMemcpyDeviceToHost, s));
    HM_CUDA_CHECK(cudaMemcpyAsync(h_tp.data(), tr->adm_tp.p, sizeof(int32_t) * na, cudaMemcpyDeviceToHost, s));
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
    // the blocks to approximate: the matrix is symmetric, so of a pair of
    // blocks with swapped ranges only the one above the diagonal
    std::vector<int32_t> upper;
    upper.reserve(na);
    int max_m_big = 1, max_n_big = 1;
    for (int64_t b = 0; b < na; ++b) {
        max_m_big = std::max(max_m_big, h_adm[4 * b + 1] - h_adm[4 * b]);
        max_n_big = std::max(max_n_big, h_adm[4 * b + 3] - h_adm[4 * b + 2]);
        if (h_tp[b] >= 0 && h_adm[4 * b] > h_adm[4 * b + 2]) continue;
        upper.push_back((int32_t)b);
    }
    auto msum = [&](int32_t b) { return h_adm[4 * b + 1] - h_adm[4 * b] + h_adm[4 * b + 3] - h_adm[4 * b + 2]; };
    // work list for a split: blocks with both dims <= SMALL_MAX_DIM and
    // m + n <= small_sum go to single warps, the others to whole CTAs (first)
    // (huge blocks, m + n > HUGE_SUM, come first: only big_ctas CTAs hold scratch for them)
    auto split = [&](const std::vector<int32_t> &blocks, int small_sum, std::vector<int32_t> &work, int64_t &n_big,
                     int &max_sum_small, int64_t &n_huge) {
        std::vector<int32_t> huge, big, small;
        max_sum_small = 2;
        for (int32_t b : blocks) {
            const int m = h_adm[4 * b + 1] - h_adm[4 * b], n = h_adm[4 * b + 3] - h_adm[4 * b + 2];
            if (m <= SMALL_MAX_DIM && n <= SMALL_MAX_DIM && m + n <= small_sum) {
                small.push_back(b);
                max_sum_small = std::max(max_sum_small, m + n);
            } else if (m + n > HUGE_SUM) {
                huge.push_back(b);
            } else {
                big.push_back(b);
            }
        }
        n_huge = (int64_t)huge.size();
        n_big = n_huge + (int64_t)big.size();
        work = huge;
        work.insert(work.end(), big.begin(), big.end());
        work.insert(work.end(), small.begin(), small.end());
    };

    const int words_r = (max_m_big + 31) / 32, words_c = (max_n_big + 31) / 32;
    // launch configurations: CTA sizes of 64, 128 and 256 threads, each with
    // the register budget of about 100 per thread
    struct Launch {
        void (*kern)(AcaArgs);
        int nt, occ;
        size_t smem;
    };
    auto make_launch = [&](void (*kern)(AcaArgs), int nt) {
        const int warps = nt / 32;
        const size_t smem_big = sizeof(double) * (32 + MAX_KMAX) + sizeof(uint32_t) * (words_r + words_c + 1) +
                                sizeof(float) * (warps + 1) * NORM_STRIDE;
        const size_t smem_small = (size_t)warps * sizeof(double) * WARP_SMEM_DOUBLES;
        Launch L{kern, nt, 0, std::max(smem_big, smem_small)};
        HM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
        HM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.occ, kern, nt, L.smem));
        if (L.occ < 1) fail(HM_EINTERNAL, "ACA kernel (%d threads) does not fit on an SM", nt);
        return L;
    };
    const Launch launches[3] = {make_launch(aca_kernel<64, 10>, 64), make_launch(aca_kernel<128, 5>, 128),
                                make_launch(aca_kernel<256, 2>, 256)};
    auto launch_of = [&](int nt) -> const Launch & { return launches[nt == 64 ? 0 : nt == 256 ? 2 : 1]; };
    const int sms = num_sms();

    AcaArgs base{};
    base.pt = tr->pt.as<double>();
    base.pf = tr->pf.as<float>();
    base.npad = tr->npad;
    base.V = tr->V.as<double>();
    base.adm = tr->adm.as<int32_t>();
    base.eps = A->params.aca_eps;
    base.kmax = kmax;
    base.qp = qp;
    // per worker: U and W as float pairs, (m + n) * kmax * 8 bytes
    base.big_stride = (int64_t)(max_m_big + max_n_big) * kmax;
    base.big_words_r = words_r;
    base.big_words_c = words_c;
    // scratch of the huge blocks (it scales with the largest admissible
    // block) for a bounded number of CTAs: two per SM, fewer where that
    // exceeds a quarter of the free memory or 20 GB; every CTA holds scratch
    // for the other large blocks (m + n <= HUGE_SUM)
    int64_t huge_cap = 0;
    {
        size_t free_b = 0, total_b = 0;
        HM_CUDA_CHECK(cudaMemGetInfo(&free_b, &total_b));
        const int64_t budget = std::min<int64_t>(20LL << 30, (int64_t)(free_b / 4));
        huge_cap = std::max<int64_t>(sms, std::min<int64_t>(2 * (int64_t)sms, budget / (8 * base.big_stride)));
    }
    auto huge_ctas = [&](int grid) { return (int)std::min<int64_t>(grid, huge_cap); };
    base.med_stride = std::min<int64_t>(base.big_stride, (int64_t)HUGE_SUM * kmax);
    DBuf scr_big, scr_med;
    scr_big.alloc(sizeof(double) * base.big_stride * huge_cap);
    base.scr_big = scr_big.as<double>();

    // Autotuner of the launch: the warp / CTA split (the m + n bound of
    // warp-mode blocks), the CTA size and the CTAs per SM.  On the first
    // assembly with a given histogram of block sizes (log2 of m + n, block
    // counts to two significant digits) the candidates run the ACA of an
    // evenly spaced sample of the blocks up to the huge tier (scratch outputs, arena sized for
    // k_max, so nothing overflows), one parameter after the other (split at
    // 128 threads and full occupancy, then the CTA size, then the CTAs per
    // SM); in each the default stays unless another is more than 5 % faster.
    // The choice is kept for every later assembly with that histogram in this
    // process.
    struct Tune {
        int small_sum, nt, ctas;
    };
    static std::mutex tune_mu;
    static std::map<std::vector<int64_t>, Tune> tune_cache;
    static std::map<ArenaKey, int64_t> arena_hint;  // last used size of the factor arena
    std::vector<int64_t> key(32, 0);
    for (int32_t b : upper) {
        int lg = 0;
        while ((1 << (lg + 1)) <= msum(b)) ++lg;
        key[std::min(lg, 31)] += 1;
    }
    for (auto &c : key) {
        int64_t scale = 1;
        while (c >= 100 * scale) scale *= 10;
        c = c / scale * scale;
    }
    key.push_back(kmax);
    key.push_back((int64_t)std::llround(std::log10(A->params.aca_eps) * 4.0));
    Tune cfg{320, ACA_THREADS, launch_of(ACA_THREADS).occ};
    bool tuned = false;
    {
        std::lock_guard<std::mutex> lk(tune_mu);
        auto it = tune_cache.find(key);
        if (it != tune_cache.end()) {
            cfg = it->second;
            tuned = true;
        }
    }
    auto run = [&](const std::vector<int32_t> &blocks, const Tune &tc, int32_t *rank, int64_t *uwo, double *arena,
                   int64_t cap, unsigned long long *ctr4, DBuf &scr_small, DBuf &d_work, AcaArgs *used) -> float {
        const Launch &L = launch_of(tc.nt);
        const int grid = sms * std::min(tc.ctas, L.occ);
        std::vector<int32_t> work;
        int64_t n_big = 0, n_huge = 0;
        int max_sum_small = 2;
        split(blocks, tc.small_sum, work, n_big, max_sum_small, n_huge);
        AcaArgs a = base;
        a.n_huge = n_huge;
        a.big_ctas = huge_ctas(grid);
        scr_med.alloc(sizeof(double) * base.med_stride * grid);
        a.scr_med = scr_med.as<double>();
        d_work.alloc(sizeof(int32_t) * std::max<size_t>(work.size(), 1));
        HM_CUDA_CHECK(cudaMemcpyAsync(d_work.p, work.data(), sizeof(int32_t) * work.size(), cudaMemcpyHostToDevice, s));
        a.work = d_work.as<int32_t>();
        a.n_big = n_big;
        a.n_work = (int64_t)work.size();
        a.small_stride = ((int64_t)max_sum_small * kmax * 3 + 1) / 2;  // U, W in FP64 + FP32 shadows
        scr_small.alloc(sizeof(double) * a.small_stride * grid * (tc.nt / 32));
        a.scr_small = scr_small.as<double>();
        a.arena_top = ctr4;
        a.q_big = ctr4 + 1;
        a.q_small = ctr4 + 2;
        a.kmax_hit = reinterpret_cast<int *>(ctr4 + 3);
        a.q_huge = ctr4 + 4;
        a.rank = rank;
        a.uw_off = uwo;
        a.arena = arena;
        a.arena_cap = cap;
        a.todo = nullptr;
        a.n_todo = 0;
        HM_CUDA_CHECK(cudaMemsetAsync(ctr4, 0, sizeof(unsigned long long) * 5, s));
        cudaEvent_t t0, t1;
        HM_CUDA_CHECK(cudaEventCreate(&t0));
        HM_CUDA_CHECK(cudaEventCreate(&t1));
        HM_CUDA_CHECK(cudaEventRecord(t0, s));
        {
            Trace trace("aca_kernel", s);
            L.kern<<<grid, L.nt, L.smem, s>>>(a);
            HM_LAUNCH_CHECK();
        }
        HM_CUDA_CHECK(cudaEventRecord(t1, s));
        HM_CUDA_CHECK(cudaEventSynchronize(t1));
        float ms = 0.0f;
        HM_CUDA_CHECK(cudaEventElapsedTime(&ms, t0, t1));
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        if (used) *used = a;
        return ms;
    };
    if (!tuned) {
        // the sample leaves out the huge blocks (m + n > HUGE_SUM): a handful
        // of them would make the sample's time the time of its longest block
        // (one CTA each), not the throughput the launch parameters decide
        std::vector<int32_t> pool;
        pool.reserve(upper.size());
        for (int32_t b : upper)
            if (msum(b) <= HUGE_SUM) pool.push_back(b);
        const size_t target = 30000;
        const size_t step = std::max<size_t>(1, pool.size() / target);
        std::vector<int32_t> sample;
        int64_t sum_mn = 0;
        for (size_t i = 0; i < pool.size(); i += step) {
            sample.push_back(pool[i]);
            sum_mn += msum(pool[i]);
        }
        if (sample.size() < pool.size() / 2 && sample.size() >= 1000) {
            DBuf t_rank, t_uwo, t_arena, t_ctr, t_scr, t_work;
            t_rank.alloc(sizeof(int32_t) * na);
            t_uwo.alloc(sizeof(int64_t) * na);
            t_arena.alloc(sizeof(double) * sum_mn * kmax);
            t_ctr.alloc(sizeof(unsigned long long) * 5);
            auto time_of = [&](const Tune &tc) {
                return run(sample, tc, t_rank.as<int32_t>(), t_uwo.as<int64_t>(), t_arena.as<double>(),
                           sum_mn * kmax, t_ctr.as<unsigned long long>(), t_scr, t_work, nullptr);
            };
            // one parameter at a time; the current value stays unless another
            // is more than 5 % faster (differences below that are timing
            // noise, and a stable choice keeps the factors identical from
            // process to process)
            auto pick = [&](std::vector<Tune> cands) {
                float t_cur = time_of(cfg);
                Tune best = cfg;
                float t_best = t_cur;
                for (const Tune &c : cands) {
                    const float t = time_of(c);
                    if (t < t_best && t < 0.95f * t_cur) {
                        best = c;
                        t_best = t;
                    }
                }
                cfg = best;
            };
            pick({Tune{160, cfg.nt, cfg.ctas}, Tune{512, cfg.nt, cfg.ctas}});
            pick({Tune{cfg.small_sum, 64, launch_of(64).occ}, Tune{cfg.small_sum, 256, launch_of(256).occ}});
            std::vector<Tune> fewer;
            for (int c = launch_of(cfg.nt).occ - 1; c >= std::max(1, launch_of(cfg.nt).occ - 2); --c)
                fewer.push_back(Tune{cfg.small_sum, cfg.nt, c});
            if (!fewer.empty()) pick(fewer);
        }
        std::lock_guard<std::mutex> lk(tune_mu);
        tune_cache[key] = cfg;
    }
    const int small_sum = cfg.small_sum;
    A->info.aca_small_sum = small_sum;
    A->info.aca_threads = cfg.nt;
    A->info.aca_ctas_per_sm = std::min(cfg.ctas, launch_of(cfg.nt).occ);
    HM_CUDA_CHECK(cudaMemsetAsync(uw_off.p, 0, sizeof(int64_t) * na, s));
    HM_CUDA_CHECK(cudaMemsetAsync(A->rank.p, 0, sizeof(int32_t) * na, s));
    // arena: sum over the approximated blocks of (m + n) * k_guess, or the size
    // the last assembly with the same blocks and tolerance used (+ 1/16), grown
    // and the overflowed blocks re-run if needed (an arena of tens of GB beyond
    // the block cache costs its mapping and unmapping on every assembly)
    int64_t upper_sum = 0;
    for (int32_t b : upper) upper_sum += msum(b);
    int64_t cap = std::max<int64_t>(upper_sum * std::min<int64_t>(kmax, 20), 1);
    const ArenaKey akey{na, upper_sum, A->params.aca_eps, kmax};
    {
        std::lock_guard<std::mutex> lk(tune_mu);
        auto it = arena_hint.find(akey);
        if (it != arena_hint.end()) cap = std::min<int64_t>(cap, it->second + it->second / 16 + 1024);
    }
    DBuf arena, ctr, scr_small, d_work;
    arena.alloc(sizeof(double) * cap);
    ctr.alloc(sizeof(unsigned long long) * 5);
    // the arguments of that run are kept for an overflow re-run
    AcaArgs a{};
    const float ms = run(upper, cfg, A->rank.as<int32_t>(), uw_off.as<int64_t>(), arena.as<double>(), cap,
                         ctr.as<unsigned long long>(), scr_small, d_work, &a);
    *sec = ms * 1e-3;
    const Launch &LL = launch_of(cfg.nt);
    const int grid = sms * std::min(cfg.ctas, LL.occ);
    unsigned long long top = read_scalar(a.arena_top, s);
    if ((int64_t)top > cap) {
        // grow: keep what fits, re-run the blocks that did not fit (CTA-wide)
        DBuf list, cnt;
        list.alloc(sizeof(int32_t) * na);
        cnt.alloc(sizeof(int));
        HM_CUDA_CHECK(cudaMemsetAsync(cnt.p, 0, sizeof(int), s));
        aca_overflow_list<<<256, 256, 0, s>>>(a.uw_off, na, list.as<int32_t>(), cnt.as<int>());
        HM_LAUNCH_CHECK();
        const int nover = read_scalar(cnt.as<int>(), s);
        // offsets only grow, so every reservation that fit ends at or below
        // cap; keep [0, cap) and restart the bump pointer there
        const int64_t used = cap;
        const int64_t newcap = (int64_t)top + (int64_t)top / 8 + 1;
        DBuf grown;
        grown.alloc(sizeof(double) * newcap);
        HM_CUDA_CHECK(cudaMemcpyAsync(grown.p, arena.p, sizeof(double) * used, cudaMemcpyDeviceToDevice, s));
        arena = std::move(grown);
        a.arena = arena.as<double>();
        a.arena_cap = newcap;
        a.todo = list.as<int32_t>();
        a.n_todo = nover;
        unsigned long long used_u = (unsigned long long)used;
        HM_CUDA_CHECK(cudaMemcpyAsync(a.arena_top, &used_u, sizeof(used_u), cudaMemcpyHostToDevice, s));
        HM_CUDA_CHECK(cudaMemsetAsync(a.q_huge, 0, sizeof(unsigned long long), s));
        Trace trace("aca_kernel", s);
        LL.kern<<<grid, LL.nt, LL.smem, s>>>(a);
        HM_LAUNCH_CHECK();
        top = read_scalar(a.arena_top, s);
        if ((int64_t)top > newcap) fail(HM_ENOMEM, "ACA factor arena overflow after growth");
    }
    // the factors stay in the arena (read once by the panel packing, then freed)
    const int64_t used = (int64_t)top;
    A->info.aca_entries = used;
    {
        std::lock_guard<std::mutex> lk(tune_mu);
        arena_hint[akey] = used;
    }
    uw = std::move(arena);
    mirror_rank_kernel<<<256, 256, 0, s>>>(tr->adm.as<int32_t>(), tr->adm_tp.as<int32_t>(), na, A->rank.as<int32_t>(),
                                           uw_off.as<int64_t>());
    HM_LAUNCH_CHECK();
    {
        // stored factor entries of the operator: sum_b k_b (m_b + n_b) over all blocks
        DBuf sz;
        sz.alloc(sizeof(int64_t) * (na + 1));
        lr_size_kernel<<<256, 256, 0, s>>>(tr->adm.as<int32_t>(), A->rank.as<int32_t>(), na, 0, sz.as<int64_t>());
        HM_LAUNCH_CHECK();
        A->lr_entries = exclusive_scan_i64(sz.as<int64_t>(), sz.as<int64_t>(), na, s);
        lr_size_kernel<<<256, 256, 0, s>>>(tr->adm.as<int32_t>(), A->rank.as<int32_t>(), na, 1, sz.as<int64_t>());
        HM_LAUNCH_CHECK();
        A->info.u_entries = exclusive_scan_i64(sz.as<int64_t>(), sz.as<int64_t>(), na, s);
    }
    // t offsets (prefix sum of ranks)
    rank_to_i64<<<256, 256, 0, s>>>(A->rank.as<int32_t>(), na, A->t_off.as<int64_t>());
    HM_LAUNCH_CHECK();
    HM_CUDA_CHECK(cudaMemsetAsync(A->t_off.as<int64_t>() + na, 0, sizeof(int64_t), s));
    A->total_rank = exclusive_scan_i64(A->t_off.as<int64_t>(), A->t_off.as<int64_t>(), na + 1, s);
    {
        DBuf st;
        st.alloc(sizeof(unsigned long long) * 2);
        HM_CUDA_CHECK(cudaMemsetAsync(st.p, 0, sizeof(unsigned long long) * 2, s));
        rank_stats<<<256, 256, 0, s>>>(A->rank.as<int32_t>(), na, st.as<unsigned long long>(),
                                       reinterpret_cast<int *>(st.as<unsigned long long>() + 1));
        HM_LAUNCH_CHECK();
        unsigned long long h[2];
        HM_CUDA_CHECK(cudaMemcpyAsync(h, st.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        HM_CUDA_CHECK(cudaStreamSynchronize(s));
        A->info.mean_rank = (double)h[0] / (double)na;
        A->info.max_rank = (int)(h[1] & 0xffffffffu);
        A->info.kmax_hit = read_scalar(a.kmax_hit, s);
    }
}

}  // namespace hm
