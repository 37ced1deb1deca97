// mv_kernels.cuh -- the streaming kernels of the H-matrix-vector product
// (Sec. 2.3): col_kernel (x_kappa^T times the W panel of each leaf column
// cluster), tsum_kernel (t_b from those partials) and row_kernel (near-field
// and U panels of each leaf row cluster against the gathered x and t).
// Included by matvec.cu only; kept apart so that a profile of these kernels
// can be tied to this file's contents.
#pragma once

#include <cuda_bf16.h>

#include "hm_internal.cuh"

namespace hm {
template <class T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

template <class T> __device__ __forceinline__ typename Acc<T>::type ld_el(const T *p) { return to_f<T>(*p); }
template <> __device__ __forceinline__ double ld_el<double>(const double *p) { return *p; }

template <class A> __device__ __forceinline__ A warp_reduce(A v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// 16-byte vector loads of panel rows (rows start on 16-byte boundaries)
// ---------------------------------------------------------------------------
template <class T> struct V16;
template <> struct V16<double> {
    static constexpr int N = 2;
    __device__ __forceinline__ static void load(const double *p, double (&v)[2]) {
        const double2 d = __ldg(reinterpret_cast<const double2 *>(p));
        v[0] = d.x;
        v[1] = d.y;
    }
};
template <> struct V16<float> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void load(const float *p, float (&v)[4]) {
        const float4 d = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = d.x;
        v[1] = d.y;
        v[2] = d.z;
        v[3] = d.w;
    }
};
template <> struct V16<__nv_bfloat16> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16 *p, float (&v)[8]) {
        const uint4 d = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[2 * q] = __uint_as_float(w[q] << 16);
            v[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
        }
    }
};

// N consecutive column indices (N * 4 bytes, aligned like the values)
template <int N> __device__ __forceinline__ void ld_idx(const int32_t *p, int (&o)[N]);
template <> __device__ __forceinline__ void ld_idx<2>(const int32_t *p, int (&o)[2]) {
    const int2 v = __ldg(reinterpret_cast<const int2 *>(p));
    o[0] = v.x;
    o[1] = v.y;
}
template <> __device__ __forceinline__ void ld_idx<4>(const int32_t *p, int (&o)[4]) {
    const int4 v = __ldg(reinterpret_cast<const int4 *>(p));
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
template <> __device__ __forceinline__ void ld_idx<8>(const int32_t *p, int (&o)[8]) {
    const int4 v = __ldg(reinterpret_cast<const int4 *>(p)), w = __ldg(reinterpret_cast<const int4 *>(p + 4));
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
    o[4] = w.x;
    o[5] = w.y;
    o[6] = w.z;
    o[7] = w.w;
}

// ---------------------------------------------------------------------------
// Phase A, t_b = W_b^T x_sigma, in two steps:
//  col_kernel : one CTA per leaf column cluster kappa computes the row vector
//               x_kappa^T Wt_kappa of kappa's column panel (the rows of every
//               W_b whose columns cover kappa, side by side): each thread owns
//               16 bytes of columns and accumulates over the |kappa| rows in
//               registers, so every thread keeps |kappa| independent 16-byte
//               loads in flight and no reduction is needed.
//  tsum_kernel: t_b(l) = sum over the column clusters of sigma_b of those
//               partials, in increasing cluster order (fixed order).
// ---------------------------------------------------------------------------
constexpr int COL_THREADS = 256;

template <class TF, class TX, class TP>
__global__ void __launch_bounds__(COL_THREADS) col_kernel(const int32_t *__restrict__ leaf_begin,
                                                          const int64_t *__restrict__ wp_off,
                                                          const int32_t *__restrict__ wp_K,
                                                          const int64_t *__restrict__ wp_colptr,
                                                          const TF *__restrict__ wp, const TX *__restrict__ x,
                                                          TP *__restrict__ p, const int32_t *__restrict__ order) {
    using A = typename Acc<TF>::type;
    constexpr int N = V16<TF>::N;
    __shared__ A s_x[MAX_LEAF];
    const int64_t kap = order ? order[blockIdx.x] : blockIdx.x;  // largest panels first
    const int32_t c0 = leaf_begin[kap], mc = leaf_begin[kap + 1] - c0;
    for (int j = threadIdx.x; j < mc; j += COL_THREADS) s_x[j] = (A)x[c0 + j];
    __syncthreads();
    const int Kw = wp_K[kap];
    const TF *W = wp + wp_off[kap];
    TP *out = p + wp_colptr[kap];
    const int nv = Kw / N;
    for (int v = threadIdx.x; v < nv; v += COL_THREADS) {
        A acc[N];
#pragma unroll
        for (int e = 0; e < N; ++e) acc[e] = 0;
        const TF *col = W + (int64_t)v * N;
        int j = 0;
        for (; j + 3 < mc; j += 4) {
            A w0[N], w1[N], w2[N], w3[N];
            V16<TF>::load(col + (int64_t)j * Kw, w0);
            V16<TF>::load(col + (int64_t)(j + 1) * Kw, w1);
            V16<TF>::load(col + (int64_t)(j + 2) * Kw, w2);
            V16<TF>::load(col + (int64_t)(j + 3) * Kw, w3);
#pragma unroll
            for (int e = 0; e < N; ++e) {
                acc[e] += w0[e] * s_x[j];
                acc[e] += w1[e] * s_x[j + 1];
                acc[e] += w2[e] * s_x[j + 2];
                acc[e] += w3[e] * s_x[j + 3];
            }
        }
        for (; j < mc; ++j) {
            A w0[N];
            V16<TF>::load(col + (int64_t)j * Kw, w0);
#pragma unroll
            for (int e = 0; e < N; ++e) acc[e] += w0[e] * s_x[j];
        }
#pragma unroll
        for (int e = 0; e < N; ++e) out[v * N + e] = (TP)acc[e];
    }
}

// t_b(l) = sum over the column clusters of sigma_b of the partials, in
// increasing cluster order.  One warp per 32 consecutive entries of t
// (coalesced stores, every lane busy whatever the ranks): b0[c] is the block
// holding entry 32 c, the lanes load the offsets t_off of the 32 blocks from
// there and each entry finds its block by a 5-step search over them (an
// entry the window does not reach, possible only after blocks of rank 0,
// searches t_off itself); the partial loads of one entry are independent
// (four accumulators, added in a fixed order).
template <class TP, class TT>
__global__ void __launch_bounds__(256) tsum_kernel(int64_t na, int64_t nt, const int32_t *__restrict__ b0tab,
                                                   const int64_t *__restrict__ t_off,
                                                   const int64_t *__restrict__ bcolptr,
                                                   const int64_t *__restrict__ pofs, const TP *__restrict__ p,
                                                   TT *__restrict__ t) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunk = (nt + 31) / 32;
    for (int64_t c = w0; c < nchunk; c += nw) {
        const int64_t b0 = b0tab[c];
        const int64_t bl = min(b0 + lane, na);
        const int64_t to = t_off[bl];  // t_off has na + 1 entries
        const int64_t e = c * 32 + lane;
        int j = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int64_t tj = __shfl_sync(full, to, j + st);
            if (tj <= e) j += st;
        }
        const int64_t to31 = __shfl_sync(full, to, 31);
        if (e >= nt) continue;
        int64_t b = b0 + j;
        if (to31 <= e && b0 + 31 < na) {
            // beyond the window: last block with t_off <= e
            int64_t lo = b0 + 31, hi = na;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (t_off[mid] <= e) lo = mid;
                else hi = mid;
            }
            b = lo;
        }
        const int l = (int)(e - t_off[b]);
        const int64_t qa = bcolptr[b], qb = bcolptr[b + 1];
        TP a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int64_t q = qa;
        for (; q + 3 < qb; q += 4) {
            a0 += p[pofs[q] + l];
            a1 += p[pofs[q + 1] + l];
            a2 += p[pofs[q + 2] + l];
            a3 += p[pofs[q + 3] + l];
        }
        for (; q < qb; ++q) a0 += p[pofs[q] + l];
        t[e] = (TT)((a0 + a1) + (a2 + a3));
    }
}

// b0[c] = the block whose t range holds entry 32 c
__global__ void tsum_b0_kernel(int64_t na, const int64_t *__restrict__ t_off, int32_t *__restrict__ b0) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = t_off[b], hi = t_off[b + 1];
        for (int64_t c = (lo + 31) / 32; c * 32 < hi; ++c) b0[c] = (int32_t)b;
    }
}

// ---------------------------------------------------------------------------
// y_rho = P_rho x(colidx) + Ut_rho t(tidx): one CTA per leaf row cluster,
// dispatched in decreasing order of panel work (`order`), so the longest
// CTAs start first and the last wave is made of short ones.
// Every row of a panel multiplies the same gathered vector, so the CTA
// gathers it once per column chunk into shared memory; then each warp takes
// RB rows at a time and streams them with 16-byte loads against the staged
// chunk (one shared-memory vector feeds RB independent global loads).
// ---------------------------------------------------------------------------
constexpr int ROW_THREADS = 256;
constexpr int ROW_WARPS = ROW_THREADS / 32;
constexpr int ROW_CHUNK = 4096;  // columns staged per pass (multiple of 8)
// Rows per warp per pass (RB): a row group is RB * ROW_WARPS rows.  The host
// picks the smallest RB whose group covers the largest leaf cluster, so the
// gathered vector is staged once per chunk and every warp keeps RB 16-byte
// loads in flight per step; rows past the cluster's end issue no loads.
// Leaves of 80 rows take two groups of 40 (RB = 5, 80 registers): measured
// on the level-8 sphere (FP64 product) 16.0 ms against 16.4 ms with one
// group of 80 (RB = 10) and 21.7 ms with RB = 12 (128 registers, 96-row
// groups); the row sums are the same bit for bit.
constexpr int row_rb_for(int max_leaf) {
    return max_leaf <= 32 ? 4 : max_leaf <= 40 ? 5 : max_leaf <= 64 ? 8 : max_leaf <= 80 ? 5 : 12;
}

// Partial sums (per lane) of rows g0 + warp + ROW_WARPS * u, u < RB, of a
// row-major panel P (|rho| x L) times z(idx), staging z(idx) chunk by chunk.
template <int RB, class T, class Z, class A>
__device__ __forceinline__ void panel_rows(const T *__restrict__ P, int L, const int32_t *__restrict__ idx,
                                           const Z *__restrict__ z, int mr, int g0, A *s_z, A (&a)[RB]) {
    constexpr int N = V16<T>::N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T *rows[RB];
    bool live[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
        const int r = g0 + warp + ROW_WARPS * u;
        live[u] = r < mr;
        rows[u] = P + (int64_t)(live[u] ? r : 0) * L;
        a[u] = 0;
    }
    for (int c0 = 0; c0 < L; c0 += ROW_CHUNK) {
        const int cl = min(ROW_CHUNK, L - c0);
        __syncthreads();
        for (int k = threadIdx.x; k < cl; k += ROW_THREADS) s_z[k] = (A)z[idx[c0 + k]];
        __syncthreads();
        const int nv = cl / N;
        // two steps in flight for FP64 panels (measured faster there; the
        // FP32 / BF16 panels are faster without)
        constexpr int UNR = sizeof(T) == 8 ? 2 : 1;
#pragma unroll UNR
        for (int v = lane; v < nv; v += 32) {
            A zv[N];
#pragma unroll
            for (int e = 0; e < N; ++e) zv[e] = s_z[v * N + e];
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                if (!live[u]) continue;
                A pv[N];
                V16<T>::load(rows[u] + c0 + (int64_t)v * N, pv);
#pragma unroll
                for (int e = 0; e < N; ++e) a[u] += pv[e] * zv[e];
            }
        }
    }
}

template <int RB, class TD, class TF, class TX, class TT, bool ORD>
__global__ void __launch_bounds__(ROW_THREADS) row_kernel(
    const int32_t *__restrict__ leaf_begin, const int64_t *__restrict__ rho_off, const int32_t *__restrict__ rho_K,
    const int64_t *__restrict__ rho_colptr, const int32_t *__restrict__ colidx, const TD *__restrict__ dense,
    const int64_t *__restrict__ up_off, const int32_t *__restrict__ up_K, const int64_t *__restrict__ up_colptr,
    const int32_t *__restrict__ tidx, const TF *__restrict__ up, const TT *__restrict__ t, const TX *__restrict__ x,
    double *__restrict__ ym, const int32_t *__restrict__ order) {
    using AD = typename Acc<TD>::type;
    using AF = typename Acc<TF>::type;
    __shared__ __align__(16) unsigned char s_raw[ROW_CHUNK * sizeof(AD)];
    const int64_t rho = ORD ? order[blockIdx.x] : blockIdx.x;  // largest panels first (ORD)
    const int32_t r0 = leaf_begin[rho], r1 = leaf_begin[rho + 1];
    const int mr = r1 - r0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TD *P = dense + rho_off[rho];
    const int Kd = rho_K[rho];
    const int32_t *ci = colidx + rho_colptr[rho];
    const TF *Q = up + up_off[rho];
    const int Ku = up_K[rho];
    const int32_t *ti = tidx + up_colptr[rho];
    for (int g0 = 0; g0 < mr; g0 += RB * ROW_WARPS) {
        AD ad[RB];
        AF af[RB];
        panel_rows<RB, TD, TX, AD>(P, Kd, ci, x, mr, g0, reinterpret_cast<AD *>(s_raw), ad);
        panel_rows<RB, TF, TT, AF>(Q, Ku, ti, t, mr, g0, reinterpret_cast<AF *>(s_raw), af);
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            const int r = g0 + warp + ROW_WARPS * u;
            const AD d = warp_reduce(ad[u]);
            const AF f = warp_reduce(af[u]);
            if (lane == 0 && r < mr) ym[r0 + r] = (double)d + (double)f;
        }
    }
}

}  // namespace hm
