// mrhs.cu -- H-matrix product with 16 right-hand sides at once on the tensor
// cores (the multi-RHS form of the H-matvec of Sec. 2.3).
//
// With one right-hand side the product reads every stored entry for one
// multiply-add (HBM-bound, CUDA cores).  With 16 it is 16 multiply-adds per
// entry: 32 flops per 4-byte near-field entry and per 2-byte BF16 factor
// entry, above what the FP32 CUDA cores deliver at HBM speed, so the three
// passes of the product become small GEMMs on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation):
//   col_bcp_kernel  : t_b (k_b x 16) = W_b^T X_sigma for every block, from
//                     the W factors regrouped by block column cluster sigma
//                     (one panel |sigma| x K_sigma per cluster, so t needs no
//                     partial sums): per tile of 64 panel columns, A = X^T
//                     from shared memory, B = panel tile staged by cp.async
//                     and read with ldmatrix.trans;
//   row_mrhs_kernel : Y_rho (|rho| x 16) = P_rho X(colidx) + U~_rho T(tidx)
//                     per leaf row cluster (A = panel rows loaded straight
//                     from HBM with 16-byte loads, B = gathered rows staged in
//                     shared memory), split over K across the 8 warps and
//                     added in a fixed order.
// Operands that are not BF16 (the FP32 near field, FP32 factors, the
// right-hand sides) are split as a = a_hi + a_lo with a_hi = bf16(a),
// a_lo = bf16(a - a_hi); a product uses hi*hi + hi*lo + lo*hi, which keeps
// about 16 significant bits (relative error ~2^-16), enough for the inner
// solves of the refinement (tolerance 1e-4).  No floating-point atomics.
//
// Layout: X [n][16] FP32 and Y [n][16] FP64 in Morton order, t [K][16]
// (16 right-hand sides contiguous).
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "hm_internal.cuh"

namespace hm {

constexpr int MR = 16;  // right-hand sides of one block product

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
    // two values of consecutive k; the lower k goes to the low half
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void split_bf16(float a, float &h, float &l) {
    h = __bfloat162float(__float2bfloat16_rn(a));
    l = a - h;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x2_trans(uint32_t &r0, uint32_t &r1, const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool pred) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
    const int n = pred ? 16 : 0;  // zero-fill when not loading
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(a), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr int CM_THREADS = 256;
constexpr int CM_COLS = 64;                 // panel columns per tile


// ---------------------------------------------------------------------------
// row_mrhs_kernel: Y_rho = P_rho X(colidx) + U~_rho T(tidx), one CTA per leaf
// row cluster, 16 MT rows per pass.  The panels are walked in slices of 16 KG
// columns through a cp.async pipeline of ST stages: the slice's panel rows and
// its gathered rows of X / T (as BF16 hi and lo, [column][rhs]) land in
// shared memory while the previous slices are multiplied; warp w owns the 16
// columns 16 (w mod KG) .. of every slice (A fragments by LDS / ldmatrix, B
// fragments by ldmatrix.trans) and, with more warps than column groups, one
// part of the MT row tiles (the parts share the staged slices); the KG column
// groups' sums are added in a fixed order at the end.
// ---------------------------------------------------------------------------
constexpr int RP_APAD = 8;         // elements of padding per staged panel row
constexpr int RP_BSTRIDE = MR + 8; // bf16 per staged column of X / T (48 bytes)

// Shape of the row pass: WARPS warps per CTA, KG column groups of 16 per
// slice (slices of 16 KG panel columns), ST pipeline stages; the WARPS / KG
// warp groups split the MT row tiles.
template <int WARPS_, int KG_, int ST_> struct RpCfg {
    static constexpr int WARPS = WARPS_, THREADS = 32 * WARPS_, KG = KG_, KS = 16 * KG_, STAGES = ST_;
    static constexpr int MG = WARPS_ / KG_;                         // warp groups over the row tiles
    static constexpr int NJ = (4 * KS + THREADS - 1) / THREADS;    // gathered 16-byte pieces per thread
    template <int MT> static constexpr int mth() { return (MT + MG - 1) / MG; }  // row tiles per warp
};

__device__ __forceinline__ void ldmatrix_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

template <int MT, class TP, class C> struct RpStage {
    static constexpr int A_BYTES = 16 * MT * (C::KS + RP_APAD) * (int)sizeof(TP);
    static constexpr int B_BYTES = 2 * C::KS * RP_BSTRIDE * 2;
    static constexpr int BYTES = A_BYTES + B_BYTES;
};

// the gathered row indices this thread needs for the slice at column c0
// (columns (tid >> 2) + (THREADS / 4) j), loaded ahead of their use
template <class C>
__device__ __forceinline__ void rp_idx(const int32_t *__restrict__ idx, int K, int c0, int (&ir)[C::NJ]) {
#pragma unroll
    for (int j = 0; j < C::NJ; ++j) {
        const int c = (threadIdx.x >> 2) + (C::THREADS / 4) * j, col = c0 + c;
        ir[j] = c < C::KS && col < K ? __ldg(idx + col) : 0;
    }
}

template <int MT, class TP, class C>
__device__ __forceinline__ void rp_load(unsigned char *stage, const TP *__restrict__ Pn, int K, int rows_valid, int c0,
                                        const int (&ir)[C::NJ], const __nv_bfloat16 *__restrict__ Zh,
                                        const __nv_bfloat16 *__restrict__ Zl) {
    TP *sA = reinterpret_cast<TP *>(stage);
    __nv_bfloat16 *sBh = reinterpret_cast<__nv_bfloat16 *>(stage + RpStage<MT, TP, C>::A_BYTES);
    __nv_bfloat16 *sBl = sBh + C::KS * RP_BSTRIDE;
    constexpr int PER = 16 / (int)sizeof(TP);  // elements per 16-byte copy
    constexpr int VPR = C::KS / PER;           // copies per row
    for (int e = threadIdx.x; e < 16 * MT * VPR; e += C::THREADS) {
        const int r = e / VPR, v = e - (e / VPR) * VPR;
        const int col = c0 + PER * v;
        const bool ok = r < rows_valid && col < K;
        cp_async16(sA + r * (C::KS + RP_APAD) + PER * v, ok ? (const void *)(Pn + (int64_t)r * K + col) : (const void *)Pn,
                   ok);
    }
#pragma unroll
    for (int j = 0; j < C::NJ; ++j) {
        const int c = (threadIdx.x >> 2) + (C::THREADS / 4) * j, q = threadIdx.x & 3;  // q: hi / lo x first / second 8 rhs
        if (c >= C::KS) continue;
        const int col = c0 + c;
        const bool ok = col < K;
        const __nv_bfloat16 *src = ((q & 2) ? Zl : Zh) + (int64_t)ir[j] * MR + 8 * (q & 1);
        __nv_bfloat16 *dst = ((q & 2) ? sBl : sBh) + c * RP_BSTRIDE + 8 * (q & 1);
        cp_async16(dst, ok ? (const void *)src : (const void *)Zh, ok);
    }
}

template <int MT, class TP, class C>
__device__ __forceinline__ void rp_compute(const unsigned char *stage, float (&acc)[C::template mth<MT>()][2][4]) {
    constexpr int MTH = C::template mth<MT>();
    const TP *sA = reinterpret_cast<const TP *>(stage);
    const __nv_bfloat16 *sBh = reinterpret_cast<const __nv_bfloat16 *>(stage + RpStage<MT, TP, C>::A_BYTES);
    const __nv_bfloat16 *sBl = sBh + C::KS * RP_BSTRIDE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int kb = 16 * (warp % C::KG), mt0 = MTH * (warp / C::KG);
    uint32_t bh[2][2], bl[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        ldmatrix_x2_trans(bh[nt][0], bh[nt][1], sBh + (kb + (lane & 15)) * RP_BSTRIDE + 8 * nt);
        ldmatrix_x2_trans(bl[nt][0], bl[nt][1], sBl + (kb + (lane & 15)) * RP_BSTRIDE + 8 * nt);
    }
#pragma unroll
    for (int ml = 0; ml < MTH; ++ml) {
        const int mt = mt0 + ml;
        if (MTH != MT && mt >= MT) break;
        if constexpr (sizeof(TP) == 4) {
            const float *r0 = reinterpret_cast<const float *>(sA) + (16 * mt + g) * (C::KS + RP_APAD) + kb + 2 * t;
            const float *r1 = r0 + 8 * (C::KS + RP_APAD);
            const float2 p0 = *reinterpret_cast<const float2 *>(r0), p1 = *reinterpret_cast<const float2 *>(r0 + 8);
            const float2 q0 = *reinterpret_cast<const float2 *>(r1), q1 = *reinterpret_cast<const float2 *>(r1 + 8);
            float h[8], l[8];
            split_bf16(p0.x, h[0], l[0]);
            split_bf16(p0.y, h[1], l[1]);
            split_bf16(q0.x, h[2], l[2]);
            split_bf16(q0.y, h[3], l[3]);
            split_bf16(p1.x, h[4], l[4]);
            split_bf16(p1.y, h[5], l[5]);
            split_bf16(q1.x, h[6], l[6]);
            split_bf16(q1.y, h[7], l[7]);
            // A regs: (row g, k 2t..), (row g+8, k 2t..), (row g, k 2t+8..), (row g+8, k 2t+8..)
            const uint32_t ah0 = pack_bf16(h[0], h[1]), ah1 = pack_bf16(h[2], h[3]), ah2 = pack_bf16(h[4], h[5]),
                           ah3 = pack_bf16(h[6], h[7]);
            const uint32_t al0 = pack_bf16(l[0], l[1]), al1 = pack_bf16(l[2], l[3]), al2 = pack_bf16(l[4], l[5]),
                           al3 = pack_bf16(l[6], l[7]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                mma_bf16(acc[ml][nt], ah0, ah1, ah2, ah3, bh[nt][0], bh[nt][1]);
                mma_bf16(acc[ml][nt], ah0, ah1, ah2, ah3, bl[nt][0], bl[nt][1]);
                mma_bf16(acc[ml][nt], al0, al1, al2, al3, bh[nt][0], bh[nt][1]);
            }
        } else {
            // ldmatrix.x4: matrices (rows 0-7, k 0-7), (rows 8-15, k 0-7), (rows 0-7, k 8-15), (rows 8-15, k 8-15)
            const __nv_bfloat16 *base = reinterpret_cast<const __nv_bfloat16 *>(sA) +
                                        (16 * mt + (lane & 15)) * (C::KS + RP_APAD) + kb + 8 * (lane >> 4);
            uint32_t a0, a1, a2, a3;
            ldmatrix_x4(a0, a1, a2, a3, base);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                mma_bf16(acc[ml][nt], a0, a1, a2, a3, bh[nt][0], bh[nt][1]);
                mma_bf16(acc[ml][nt], a0, a1, a2, a3, bl[nt][0], bl[nt][1]);
            }
        }
    }
}

template <int MT, class TP, class C>
__device__ __forceinline__ void rp_panel(unsigned char *sm, const TP *__restrict__ Pn, int K, int rows_valid,
                                         const int32_t *__restrict__ idx, const __nv_bfloat16 *__restrict__ Zh,
                                         const __nv_bfloat16 *__restrict__ Zl,
                                         float (&acc)[C::template mth<MT>()][2][4]) {
    constexpr int SB = RpStage<MT, TP, C>::BYTES, KS = C::KS, ST = C::STAGES;
    const int ns = (K + KS - 1) / KS;
    int ir[C::NJ];
#pragma unroll
    for (int st = 0; st < ST - 1; ++st) {
        if (st < ns) {
            rp_idx<C>(idx, K, st * KS, ir);
            rp_load<MT, TP, C>(sm + st * SB, Pn, K, rows_valid, st * KS, ir, Zh, Zl);
        }
        cp_async_commit();
    }
    rp_idx<C>(idx, K, (ST - 1) * KS, ir);  // indices of the next slice to load
    for (int sl = 0; sl < ns; ++sl) {
        cp_async_wait<ST - 2>();
        __syncthreads();
        const int nx = sl + ST - 1;
        if (nx < ns) rp_load<MT, TP, C>(sm + (nx % ST) * SB, Pn, K, rows_valid, nx * KS, ir, Zh, Zl);
        cp_async_commit();
        rp_idx<C>(idx, K, (nx + 1) * KS, ir);  // consumed one iteration later
        rp_compute<MT, TP, C>(sm + (sl % ST) * SB, acc);
    }
    cp_async_wait<0>();
    __syncthreads();
}

// Output of the row pass: mode 0 = Y [n][16] FP64 (Morton rows); 1 / 2 =
// the first nr columns into p as [column][ld] FP32 / FP64 (the layout of a
// block of Krylov vectors), the same values (FP32 sums, widened or not).
struct YOut {
    void *p;
    int64_t ld;
    int nr, mode;
};

// TAIL: the U panels come in two parts, the leading terms (up, TF = float)
// and the trailing ones (u16, BF16), multiplied one after the other into the
// same accumulators
template <int MT, class TF, class C, bool TAIL>
__global__ void __launch_bounds__(C::THREADS) row_mrhs_kernel(
    const int32_t *__restrict__ leaf_begin, const int64_t *__restrict__ rho_off, const int32_t *__restrict__ rho_K,
    const int64_t *__restrict__ rho_colptr, const int32_t *__restrict__ colidx, const float *__restrict__ dense,
    const int64_t *__restrict__ up_off, const int32_t *__restrict__ up_K, const int64_t *__restrict__ up_colptr,
    const int32_t *__restrict__ tidx, const TF *__restrict__ up, const int64_t *__restrict__ u16_off,
    const int32_t *__restrict__ u16_K, const int64_t *__restrict__ u16_colptr, const int32_t *__restrict__ u16_tidx,
    const __nv_bfloat16 *__restrict__ u16, const __nv_bfloat16 *__restrict__ Th,
    const __nv_bfloat16 *__restrict__ Tl, const __nv_bfloat16 *__restrict__ Xh, const __nv_bfloat16 *__restrict__ Xl,
    double *__restrict__ Y, YOut yo) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int64_t rho = blockIdx.x;
    const int32_t r0 = leaf_begin[rho], mr = leaf_begin[rho + 1] - r0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int Kd = rho_K[rho], Ku = up_K[rho];
    constexpr int MTH = C::template mth<MT>();
    const int kg = warp % C::KG, mt0 = MTH * (warp / C::KG);
    for (int r0t = 0; r0t < mr; r0t += 16 * MT) {
        const int rows = min(16 * MT, mr - r0t);
        float acc[MTH][2][4];
#pragma unroll
        for (int ml = 0; ml < MTH; ++ml)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[ml][nt][e] = 0.0f;
        rp_panel<MT, float, C>(sm, dense + rho_off[rho] + (int64_t)r0t * Kd, Kd, rows, colidx + rho_colptr[rho], Xh,
                               Xl, acc);
        rp_panel<MT, TF, C>(sm, up + up_off[rho] + (int64_t)r0t * Ku, Ku, rows, tidx + up_colptr[rho], Th, Tl, acc);
        if constexpr (TAIL) {
            const int K16 = u16_K[rho];
            rp_panel<MT, __nv_bfloat16, C>(sm, u16 + u16_off[rho] + (int64_t)r0t * K16, K16, rows,
                                           u16_tidx + u16_colptr[rho], Th, Tl, acc);
        }
        // per-column-group sums -> shared memory -> fixed-order sum over the KG groups
        float *red = reinterpret_cast<float *>(sm);
#pragma unroll
        for (int ml = 0; ml < MTH; ++ml) {
            const int mt = mt0 + ml;
            if (MTH != MT && mt >= MT) break;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                float *base = red + kg * (16 * MT) * MR;
                const int ra = 16 * mt + g, col = 8 * nt + 2 * t;
                base[ra * MR + col] = acc[ml][nt][0];
                base[ra * MR + col + 1] = acc[ml][nt][1];
                base[(ra + 8) * MR + col] = acc[ml][nt][2];
                base[(ra + 8) * MR + col + 1] = acc[ml][nt][3];
            }
        }
        __syncthreads();
        if (yo.mode == 0) {
            for (int e = threadIdx.x; e < rows * MR; e += C::THREADS) {
                float sacc = 0.0f;
                for (int w = 0; w < C::KG; ++w) sacc += red[w * (16 * MT) * MR + e];
                Y[(int64_t)(r0 + r0t) * MR + e] = (double)sacc;
            }
        } else {
            // the same sums through a [column][row] tile to the first yo.nr
            // columns of [column][ld] (one coalesced row run per column)
            constexpr int TP = 16 * MT + 1;
            float *tile = red + C::KG * (16 * MT) * MR;
            for (int e = threadIdx.x; e < rows * MR; e += C::THREADS) {
                float sacc = 0.0f;
                for (int w = 0; w < C::KG; ++w) sacc += red[w * (16 * MT) * MR + e];
                tile[(e % MR) * TP + e / MR] = sacc;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < yo.nr * rows; e += C::THREADS) {
                const int col = e / rows, row = e - col * rows;
                const float v = tile[col * TP + row];
                const int64_t at = (int64_t)col * yo.ld + r0 + r0t + row;
                if (yo.mode == 1) static_cast<float *>(yo.p)[at] = v;
                else static_cast<double *>(yo.p)[at] = (double)v;
            }
        }
        __syncthreads();
    }
}

// Xh + Xl = X (BF16 pair of every FP32 value)
__global__ void split_rows_kernel(const float *__restrict__ X, int64_t n, __nv_bfloat16 *__restrict__ Xh,
                                  __nv_bfloat16 *__restrict__ Xl) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float h, l;
        split_bf16(X[e], h, l);
        Xh[e] = __float2bfloat16_rn(h);
        Xl[e] = __float2bfloat16_rn(l);
    }
}

// The same pairs straight from a block of vectors x [nr][ldx] (FP32 or FP64,
// Morton order): X[m][r] = (float) x[r][m] (0 for r >= nr), split as above,
// 64 rows per step transposed through shared memory (read along m, written
// along r)
constexpr int GS_ROWS = 64;
template <class TI>
__global__ void __launch_bounds__(256) gather_split_kernel(const TI *__restrict__ x, int64_t n, int nr, int64_t ldx,
                                                           __nv_bfloat16 *__restrict__ Xh,
                                                           __nv_bfloat16 *__restrict__ Xl) {
    __shared__ float s_x[MR][GS_ROWS + 1];
    for (int64_t i0 = blockIdx.x * (int64_t)GS_ROWS; i0 < n; i0 += (int64_t)gridDim.x * GS_ROWS) {
        const int rows = (int)((n - i0) < GS_ROWS ? (n - i0) : (int64_t)GS_ROWS);
        __syncthreads();
        for (int e = threadIdx.x; e < MR * GS_ROWS; e += blockDim.x) {
            const int r = e / GS_ROWS, i = e - r * GS_ROWS;
            s_x[r][i] = (r < nr && i < rows) ? (float)x[(int64_t)r * ldx + i0 + i] : 0.0f;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * MR; e += blockDim.x) {
            const int i = e / MR, r = e - i * MR;
            float h, l;
            split_bf16(s_x[r][i], h, l);
            Xh[(i0 + i) * MR + r] = __float2bfloat16_rn(h);
            Xl[(i0 + i) * MR + r] = __float2bfloat16_rn(l);
        }
    }
}

// ---------------------------------------------------------------------------
// col_bcp_kernel: t_b = X_sigma^T W_b for every block, straight from the
// panels grouped by block column cluster (no partial sums): one CTA per tile
// of 64 panel columns and at most BC_SPLIT panel rows (the rows of taller
// panels are split over several CTAs whose partials are added afterwards).
// ---------------------------------------------------------------------------

// one work item: (panel, first column, first row, end row, partial slot or -1)
constexpr int BC_ITEM = 5;
constexpr int BC_SPLIT = 1024;  // rows of one work item (taller panels are split, partials added after)

// the t rows of 64 panel columns as BF16 pairs (hi + lo = value)
__device__ __forceinline__ void store_t_pair(__nv_bfloat16 *Th, __nv_bfloat16 *Tl, int64_t ti, int r, float v) {
    float h, l;
    split_bf16(v, h, l);
    Th[ti * MR + r] = __float2bfloat16_rn(h);
    Tl[ti * MR + r] = __float2bfloat16_rn(l);
}

// Pipelined over chunks of BP_KC panel rows (3 stages of cp.async): the
// chunk's rows of X (pre-split BF16 pairs, [row][rhs]) and of the W tile land
// in shared memory while earlier chunks are multiplied.  A = X^T fragments by
// ldmatrix.trans from the [row][rhs] tile; B = W fragments by ldmatrix.trans
// (BF16 panels) or by shared-memory loads split into BF16 pairs (FP32
// panels).  Each of the 8 warps owns 8 of the 64 columns.
// Chunks of 16 panel rows in 6 stages (35 KB of shared memory per CTA; the
// kernel's 43 registers allow 5 CTAs of 8 warps per SM).  Measured on the
// level-8 sphere (FP32 factors, rows x stages): 64 x 3 4.70 ms, 64 x 4 5.61,
// 32 x 3 4.37, 32 x 4 4.23, 32 x 5 4.85, 32 x 6 4.83, 16 x 6 3.85, 16 x 8 4.29;
// the same t bit for bit (the k order of the MMAs does not depend on them).
constexpr int BP_KC = 16;               // panel rows per chunk
static_assert(BP_KC % 16 == 0, "bp_compute takes 16 chunk rows per MMA step");
constexpr int BP_STAGES = 6;
constexpr int BP_XSTRIDE = MR + 8;      // bf16 per staged row of X (48 bytes)
constexpr int BP_WS16 = CM_COLS + 8;    // bf16 per staged W row (144 bytes)
constexpr int BP_WS32 = CM_COLS + 4;    // floats per staged W row (conflict-free column reads)

template <class TF> struct BpStage {
    static constexpr int X_BYTES = 2 * BP_KC * BP_XSTRIDE * 2;
    static constexpr int W_BYTES = sizeof(TF) == 2 ? BP_KC * BP_WS16 * 2 : BP_KC * BP_WS32 * 4;
    static constexpr int BYTES = X_BYTES + W_BYTES;
};

template <class TF>
__device__ __forceinline__ void bp_load(unsigned char *stage, const TF *__restrict__ W, int K, int kc, int n0,
                                        const __nv_bfloat16 *__restrict__ Xh, const __nv_bfloat16 *__restrict__ Xl,
                                        int64_t xr0) {
    __nv_bfloat16 *sXh = reinterpret_cast<__nv_bfloat16 *>(stage);
    __nv_bfloat16 *sXl = sXh + BP_KC * BP_XSTRIDE;
    for (int e = threadIdx.x; e < BP_KC * 4; e += CM_THREADS) {
        const int k = e >> 2, q = e & 3;
        const bool ok = k < kc;
        const __nv_bfloat16 *src = ((q & 2) ? Xl : Xh) + (xr0 + k) * MR + 8 * (q & 1);
        cp_async16(((q & 2) ? sXl : sXh) + k * BP_XSTRIDE + 8 * (q & 1), ok ? (const void *)src : (const void *)Xh,
                   ok);
    }
    constexpr int PER = 16 / (int)sizeof(TF), VPR = CM_COLS / PER;
    constexpr int WS = sizeof(TF) == 2 ? BP_WS16 : BP_WS32;
    TF *sW = reinterpret_cast<TF *>(stage + BpStage<TF>::X_BYTES);
    for (int e = threadIdx.x; e < BP_KC * VPR; e += CM_THREADS) {
        const int k = e / VPR, v = e - (e / VPR) * VPR;
        const int col = n0 + PER * v;
        const bool ok = k < kc && col < K;
        cp_async16(sW + k * WS + PER * v, ok ? (const void *)(W + (int64_t)k * K + col) : (const void *)W, ok);
    }
}

template <class TF>
__device__ __forceinline__ void bp_compute(const unsigned char *stage, float (&d)[4]) {
    const __nv_bfloat16 *sXh = reinterpret_cast<const __nv_bfloat16 *>(stage);
    const __nv_bfloat16 *sXl = sXh + BP_KC * BP_XSTRIDE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    // ldmatrix.x4.trans of X^T: lanes 0-7 rows k 0-7 / rhs 0-7, 8-15 rows k 0-7 / rhs 8-15,
    // 16-23 rows k 8-15 / rhs 0-7, 24-31 rows k 8-15 / rhs 8-15
    const int xr = (lane & 7) + 8 * (lane >> 4), xc = 8 * ((lane >> 3) & 1);
#pragma unroll
    for (int kb = 0; kb < BP_KC; kb += 16) {
        uint32_t ah0, ah1, ah2, ah3, al0, al1, al2, al3;
        {
            const uint32_t a = (uint32_t)__cvta_generic_to_shared(sXh + (kb + xr) * BP_XSTRIDE + xc);
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                         : "=r"(ah0), "=r"(ah1), "=r"(ah2), "=r"(ah3)
                         : "r"(a));
            const uint32_t b = (uint32_t)__cvta_generic_to_shared(sXl + (kb + xr) * BP_XSTRIDE + xc);
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                         : "=r"(al0), "=r"(al1), "=r"(al2), "=r"(al3)
                         : "r"(b));
        }
        if constexpr (sizeof(TF) == 2) {
            const __nv_bfloat16 *sW = reinterpret_cast<const __nv_bfloat16 *>(stage + BpStage<TF>::X_BYTES);
            uint32_t b0, b1;
            ldmatrix_x2_trans(b0, b1, sW + (kb + (lane & 15)) * BP_WS16 + 8 * warp);
            mma_bf16(d, ah0, ah1, ah2, ah3, b0, b1);
            mma_bf16(d, al0, al1, al2, al3, b0, b1);
        } else {
            const float *sW = reinterpret_cast<const float *>(stage + BpStage<TF>::X_BYTES);
            const float *c = sW + 8 * warp + g;
            float h[4], l[4];
            split_bf16(c[(kb + 2 * t) * BP_WS32], h[0], l[0]);
            split_bf16(c[(kb + 2 * t + 1) * BP_WS32], h[1], l[1]);
            split_bf16(c[(kb + 2 * t + 8) * BP_WS32], h[2], l[2]);
            split_bf16(c[(kb + 2 * t + 9) * BP_WS32], h[3], l[3]);
            const uint32_t bh0 = pack_bf16(h[0], h[1]), bh1 = pack_bf16(h[2], h[3]);
            const uint32_t bl0 = pack_bf16(l[0], l[1]), bl1 = pack_bf16(l[2], l[3]);
            mma_bf16(d, ah0, ah1, ah2, ah3, bh0, bh1);
            mma_bf16(d, al0, al1, al2, al3, bh0, bh1);
            mma_bf16(d, ah0, ah1, ah2, ah3, bl0, bl1);
        }
    }
}

template <class TF>
__global__ void __launch_bounds__(CM_THREADS) col_bcp_kernel(const int32_t *__restrict__ items,
                                                             const int64_t *__restrict__ off,
                                                             const int32_t *__restrict__ Kg,
                                                             const int32_t *__restrict__ rows,
                                                             const int64_t *__restrict__ col0,
                                                             const int32_t *__restrict__ tidx,
                                                             const TF *__restrict__ bcp,
                                                             const __nv_bfloat16 *__restrict__ Xh,
                                                             const __nv_bfloat16 *__restrict__ Xl,
                                                             __nv_bfloat16 *__restrict__ Th,
                                                             __nv_bfloat16 *__restrict__ Tl,
                                                             float *__restrict__ part) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int32_t *it = items + BC_ITEM * (int64_t)blockIdx.x;
    const int grp = it[0], n0 = it[1], slot = it[4];
    const int32_t r0 = rows[2 * grp] + it[2], nr = it[3] - it[2];
    const int K = Kg[grp];
    const TF *W = bcp + off[grp] + (int64_t)it[2] * K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    constexpr int SB = BpStage<TF>::BYTES;
    const int ns = (nr + BP_KC - 1) / BP_KC;
    float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int st = 0; st < BP_STAGES - 1; ++st) {
        if (st < ns)
            bp_load<TF>(sm + st * SB, W + (int64_t)st * BP_KC * K, K, min(BP_KC, nr - st * BP_KC), n0, Xh, Xl,
                        r0 + st * BP_KC);
        cp_async_commit();
    }
    for (int c = 0; c < ns; ++c) {
        cp_async_wait<BP_STAGES - 2>();
        __syncthreads();
        const int nx = c + BP_STAGES - 1;
        if (nx < ns)
            bp_load<TF>(sm + (nx % BP_STAGES) * SB, W + (int64_t)nx * BP_KC * K, K, min(BP_KC, nr - nx * BP_KC), n0,
                        Xh, Xl, r0 + nx * BP_KC);
        cp_async_commit();
        bp_compute<TF>(sm + (c % BP_STAGES) * SB, d);
    }
    cp_async_wait<0>();
    // D (16 rhs x 8 columns of this warp) -> t rows of those columns, or the partial of this row range
    const int cl = 8 * warp + 2 * t, col = n0 + cl;
    if (slot >= 0) {
        float *pp = part + (int64_t)slot * CM_COLS * MR;
        pp[cl * MR + g] = d[0];
        pp[cl * MR + g + 8] = d[2];
        pp[(cl + 1) * MR + g] = d[1];
        pp[(cl + 1) * MR + g + 8] = d[3];
        return;
    }
    const int64_t cbase = col0[grp];
    if (col < K) {
        const int32_t ti = tidx[cbase + col];
        if (ti >= 0) {
            store_t_pair(Th, Tl, ti, g, d[0]);
            store_t_pair(Th, Tl, ti, g + 8, d[2]);
        }
    }
    if (col + 1 < K) {
        const int32_t ti = tidx[cbase + col + 1];
        if (ti >= 0) {
            store_t_pair(Th, Tl, ti, g, d[1]);
            store_t_pair(Th, Tl, ti, g + 8, d[3]);
        }
    }
}

// tiles whose rows were split: t = sum of the partials in row order
// (red: (panel, first column, first slot, slots) per tile)
__global__ void bcp_reduce_kernel(const int32_t *__restrict__ red, const int32_t *__restrict__ Kg,
                                  const int64_t *__restrict__ col0, const int32_t *__restrict__ tidx,
                                  const float *__restrict__ part, __nv_bfloat16 *__restrict__ Th,
                                  __nv_bfloat16 *__restrict__ Tl) {
    const int32_t *rd = red + 4 * (int64_t)blockIdx.x;
    const int grp = rd[0], n0 = rd[1], s0 = rd[2], ns = rd[3];
    const int K = Kg[grp];
    for (int e = threadIdx.x; e < CM_COLS * MR; e += blockDim.x) {
        const int cl = e / MR, r = e - (e / MR) * MR;
        if (n0 + cl >= K) continue;
        const int32_t ti = tidx[col0[grp] + n0 + cl];
        if (ti < 0) continue;
        float acc = 0.0f;
        // eight partials' loads in flight, added in row order
#pragma unroll 8
        for (int k = 0; k < ns; ++k) acc += part[((int64_t)(s0 + k) * CM_COLS + cl) * MR + r];
        store_t_pair(Th, Tl, ti, r, acc);
    }
}

// W_b into its block-column panel: for every leaf column cluster kappa of
// sigma_b, the rows of kappa come from kappa's W panel (FP64 master); b's
// position in kappa's block list (ascending) by a binary search per thread.
// rank: the terms of b in this panel set, from term lofs[b] on (lofs null:
// from the first); blocks without terms in the set have no panel columns.
template <class TF>
__global__ void bcp_pack_kernel(const int32_t *__restrict__ adm, const int32_t *__restrict__ rank,
                                const int32_t *__restrict__ lofs, const int32_t *__restrict__ bgrp,
                                const int32_t *__restrict__ bkoff,
                                const int64_t *__restrict__ off, const int32_t *__restrict__ Kg,
                                const int32_t *__restrict__ leaf_begin, int64_t nleaf,
                                const int64_t *__restrict__ lr_colptr, const int32_t *__restrict__ lr_collist,
                                const int64_t *__restrict__ wp_off, const int32_t *__restrict__ wp_K,
                                const int32_t *__restrict__ wp_koff, const double *__restrict__ wp,
                                TF *__restrict__ bcp) {
    const int32_t b = blockIdx.x;
    const int32_t cb = adm[4 * b + 2], ce = adm[4 * b + 3];
    const int k = rank[b];
    if (k == 0) return;
    const int l0 = lofs ? lofs[b] : 0;
    const int grp = bgrp[b], koff = bkoff[b], K = Kg[grp];
    TF *P = bcp + off[grp];
    // first leaf cluster of sigma_b
    int64_t lo = 0, hi = nleaf;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (leaf_begin[mid] <= cb) lo = mid;
        else hi = mid;
    }
    for (int64_t kap = lo; kap < nleaf && leaf_begin[kap] < ce; ++kap) {
        int64_t q = lr_colptr[kap], qe = lr_colptr[kap + 1];
        while (qe - q > 1) {  // last position with lr_collist <= b
            const int64_t mid = (q + qe) >> 1;
            if (lr_collist[mid] <= b) q = mid;
            else qe = mid;
        }
        if (q >= lr_colptr[kap + 1] || lr_collist[q] != b) continue;  // cannot happen for a consistent block list
        const int32_t k0 = leaf_begin[kap], mk = leaf_begin[kap + 1] - k0;
        const double *src = wp + wp_off[kap] + wp_koff[q] + l0;
        for (int e = threadIdx.x; e < mk * k; e += blockDim.x) {
            const int j = e / k, l = e - (e / k) * k;
            const double v = src[(int64_t)j * wp_K[kap] + l];
            if constexpr (sizeof(TF) == 2) P[(int64_t)(k0 - cb + j) * K + koff + l] = __double2bfloat16(v);
            else P[(int64_t)(k0 - cb + j) * K + koff + l] = (float)v;
        }
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static unsigned grid1d_m(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 65535LL * 8));
}

// X[m][r] = x_r[perm[m]] (FP32) for r < nrhs, 0 for the unused columns
__global__ void mrhs_gather_kernel(const double *__restrict__ x, int64_t n, int nrhs, const int32_t *__restrict__ perm,
                                   float *__restrict__ X) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * MR; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / MR;
        const int r = (int)(e - m * MR);
        X[e] = r < nrhs ? (float)x[(int64_t)r * n + perm[m]] : 0.0f;
    }
}

// y_r[perm[m]] = alpha Y[m][r] + beta y_r[perm[m]]
__global__ void mrhs_scatter_kernel(const double *__restrict__ Y, int64_t n, int nrhs, const int32_t *__restrict__ perm,
                                    double alpha, double beta, double *__restrict__ y) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n);
        const int64_t m = e - (int64_t)r * n;
        const int64_t i = (int64_t)r * n + perm[m];
        const double v = alpha * Y[m * MR + r];
        y[i] = beta == 0.0 ? v : v + beta * y[i];
    }
}

// sort keys of the admissible blocks: (column begin, column end) in 2 nb
// bits; blocks without terms in the panel set get the all-ones key, which no
// block's bounds make (column begins are < n < 2^nb - 1), and sort last
__global__ void bcp_keys_kernel(const int32_t *__restrict__ adm, const int32_t *__restrict__ rank, int64_t na, int nb,
                                uint64_t *__restrict__ key, int32_t *__restrict__ id) {
    const uint64_t none = (uint64_t(1) << (2 * nb)) - 1;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x) {
        key[b] = rank[b] == 0 ? none
                              : ((uint64_t)(uint32_t)adm[4 * b + 2] << nb) | (uint64_t)(uint32_t)adm[4 * b + 3];
        id[b] = (int32_t)b;
    }
}

// Grouping of the sorted admissible blocks into block-column panels, on the
// device.  A group is a run of equal keys (one column cluster); its panel
// holds the W factors of its blocks side by side in sorted order, width
// rounded up to 8 (at least 8), and is cut into work items of CM_COLS panel
// columns and at most BC_SPLIT rows (taller panels give several items whose
// partial products go to consecutive slots and are added by one reduction
// item per column tile).

// head[i] = 1 where a run of equal keys starts (0 for the blocks without
// terms and for head[na]); rk64 = the sorted ranks as int64 (rk64[na] = 0)
__global__ void bcp_head_kernel(const uint64_t *__restrict__ key, const int32_t *__restrict__ rk, int64_t na,
                                uint64_t none, int64_t *__restrict__ head, int64_t *__restrict__ rk64) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= na; i += (int64_t)gridDim.x * blockDim.x) {
        head[i] = i < na && key[i] != none && (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
        rk64[i] = i < na ? rk[i] : 0;
    }
}

// gs[g] = first sorted position of group g (from the exclusive scan of head),
// gs[ng] = the end of the last group (the first block without terms, or na)
__global__ void bcp_gstart_kernel(const uint64_t *__restrict__ key, const int64_t *__restrict__ head,
                                  const int64_t *__restrict__ gx, int64_t na, int64_t ng, uint64_t none,
                                  int64_t *__restrict__ gs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < na; i += (int64_t)gridDim.x * blockDim.x) {
        if (head[i]) gs[gx[i]] = i;
        if (key[i] == none && (i == 0 || key[i - 1] != none)) gs[ng] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && key[na - 1] != none) gs[ng] = na;
}

// per group: panel width K, rows (cb, ce), and the counts that the scans turn
// into offsets (cnt[q][g], q = panel entries, width, items, reductions, slots)
__global__ void bcp_group_kernel(const uint64_t *__restrict__ key, const int64_t *__restrict__ gs,
                                 const int64_t *__restrict__ rpre, int64_t ng, int nb, int32_t *__restrict__ Kg,
                                 int32_t *__restrict__ rows, int64_t *__restrict__ cnt) {
    const uint64_t cmask = (uint64_t(1) << nb) - 1;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g <= ng; g += (int64_t)gridDim.x * blockDim.x) {
        if (g == ng) {  // the scans' last (total) entries
            for (int q = 0; q < 5; ++q) cnt[q * (ng + 1) + ng] = 0;
            continue;
        }
        const int64_t i0 = gs[g], k = rpre[gs[g + 1]] - rpre[i0];
        const int32_t K = k <= 8 ? 8 : (int32_t)((k + 7) / 8 * 8);
        const uint64_t kk = key[i0];
        const int32_t cb = (int32_t)(kk >> nb), ce = (int32_t)(kk & cmask), nrow = ce - cb;
        const int32_t ncolt = (K + CM_COLS - 1) / CM_COLS, nsplit = (nrow + BC_SPLIT - 1) / BC_SPLIT;
        Kg[g] = K;
        rows[2 * g] = cb;
        rows[2 * g + 1] = ce;
        cnt[0 * (ng + 1) + g] = (int64_t)nrow * K;
        cnt[1 * (ng + 1) + g] = K;
        cnt[2 * (ng + 1) + g] = nsplit == 1 ? ncolt : (int64_t)ncolt * nsplit;
        cnt[3 * (ng + 1) + g] = nsplit == 1 ? 0 : ncolt;
        cnt[4 * (ng + 1) + g] = nsplit == 1 ? 0 : (int64_t)ncolt * nsplit;
    }
}

// per sorted block with terms in the set: its group, its column offset in
// the panel, and the map from its panel columns to its entries of t (the
// set's terms of b start at term lofs[b], at 0 when lofs is null)
__global__ void bcp_block_kernel(const int64_t *__restrict__ gx, const int64_t *__restrict__ head,
                                 const int64_t *__restrict__ gs, const int64_t *__restrict__ rpre,
                                 const int32_t *__restrict__ id, const int32_t *__restrict__ rk,
                                 const int32_t *__restrict__ lofs, const int64_t *__restrict__ col0,
                                 const int64_t *__restrict__ t_off, int64_t ng, int32_t *__restrict__ bgrp,
                                 int32_t *__restrict__ bkoff, int32_t *__restrict__ tidx) {
    const int64_t nend = gs[ng];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nend; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = gx[i] + head[i] - 1;
        const int32_t b = id[i], koff = (int32_t)(rpre[i] - rpre[gs[g]]);
        const int64_t t0 = t_off[b] + (lofs ? lofs[b] : 0);
        bgrp[b] = (int32_t)g;
        bkoff[b] = koff;
        int32_t *ti = tidx + col0[g] + koff;
        for (int l = 0; l < rk[i]; ++l) ti[l] = (int32_t)(t0 + l);
    }
}

// the work items (grp, first column, first row, end row, slot or -1) and the
// reduction items (grp, first column, first slot, slots), in group order and
// column-tile order within a group
__global__ void bcp_items_kernel(const int32_t *__restrict__ Kg, const int32_t *__restrict__ rows,
                                 const int64_t *__restrict__ toff, const int64_t *__restrict__ roff,
                                 const int64_t *__restrict__ soff, int64_t ng, int32_t *__restrict__ tiles,
                                 int32_t *__restrict__ red) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t K = Kg[g], nrow = rows[2 * g + 1] - rows[2 * g];
        const int32_t ncolt = (K + CM_COLS - 1) / CM_COLS, nsplit = (nrow + BC_SPLIT - 1) / BC_SPLIT;
        for (int32_t t = 0; t < ncolt; ++t) {
            const int32_t n0 = t * CM_COLS;
            if (nsplit == 1) {
                int32_t *it = tiles + BC_ITEM * (toff[g] + t);
                it[0] = (int32_t)g;
                it[1] = n0;
                it[2] = 0;
                it[3] = nrow;
                it[4] = -1;
                continue;
            }
            const int32_t s0 = (int32_t)(soff[g] + (int64_t)t * nsplit);
            int32_t *rd = red + 4 * (roff[g] + t);
            rd[0] = (int32_t)g;
            rd[1] = n0;
            rd[2] = s0;
            rd[3] = nsplit;
            for (int32_t q = 0; q < nsplit; ++q) {
                int32_t *it = tiles + BC_ITEM * (toff[g] + (int64_t)t * nsplit + q);
                it[0] = (int32_t)g;
                it[1] = n0;
                it[2] = q * BC_SPLIT;
                it[3] = (q + 1) * BC_SPLIT < nrow ? (q + 1) * BC_SPLIT : nrow;
                it[4] = s0 + q;
            }
        }
    }
}

__global__ void fill_i32_kernel(int32_t *__restrict__ a, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

// k_b - k32_b: the trailing terms of every block (BF16 tails)
__global__ void tail_rank_kernel(const int32_t *__restrict__ rank, const int32_t *__restrict__ rank32, int64_t na,
                                 int32_t *__restrict__ out) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x)
        out[b] = rank[b] - rank32[b];
}

// The block-column panels of a set of terms of the W factors (built on first
// use): blocks grouped by column cluster (sorted on the device by (column
// begin, column end), ties in block order: a stable radix sort of the block
// ids), panel widths rounded up to 8 columns; the grouping, the panels'
// offsets and the work items are computed on the device.  rk: the set's
// terms per block, from term lofs[b] on (lofs null: from the first); prec:
// the panels' type (HM_F32 or HM_BF16).
static void build_bcp(hm_matrix *A, BcpSet &S, hm_dtype prec, const int32_t *rk_set, const int32_t *lofs,
                      cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t na = tr->n_adm;
    // column bounds are <= n < 2^nb - 1
    int nb = 1;
    while (nb < 31 && (int64_t(1) << nb) <= tr->n + 1) ++nb;
    const uint64_t none = (uint64_t(1) << (2 * nb)) - 1;
    DBuf key, id, tkey, tid, rk, head, rk64, gx, rpre, gs, cnt, cx, d_bgrp, d_bkoff;
    const int64_t na1 = std::max<int64_t>(na, 1);
    key.alloc(sizeof(uint64_t) * na1);
    tkey.alloc(sizeof(uint64_t) * na1);
    id.alloc(sizeof(int32_t) * na1);
    tid.alloc(sizeof(int32_t) * na1);
    rk.alloc(sizeof(int32_t) * na1);
    head.alloc(sizeof(int64_t) * (na + 1));
    rk64.alloc(sizeof(int64_t) * (na + 1));
    gx.alloc(sizeof(int64_t) * (na + 1));
    rpre.alloc(sizeof(int64_t) * (na + 1));
    d_bgrp.alloc(sizeof(int32_t) * na1);
    d_bkoff.alloc(sizeof(int32_t) * na1);
    int64_t ng = 0;
    if (na > 0) {
        bcp_keys_kernel<<<grid1d_m(na), 256, 0, s>>>(tr->adm.as<int32_t>(), rk_set, na, nb, key.as<uint64_t>(),
                                                      id.as<int32_t>());
        HM_LAUNCH_CHECK();
        radix_sort_u64(key.as<uint64_t>(), id.as<int32_t>(), tkey.as<uint64_t>(), tid.as<int32_t>(), na, 2 * nb, s);
        gather_i32(rk_set, id.as<int32_t>(), rk.as<int32_t>(), na, s);
        bcp_head_kernel<<<grid1d_m(na + 1), 256, 0, s>>>(key.as<uint64_t>(), rk.as<int32_t>(), na, none,
                                                          head.as<int64_t>(), rk64.as<int64_t>());
        HM_LAUNCH_CHECK();
        ng = exclusive_scan_i64(head.as<int64_t>(), gx.as<int64_t>(), na + 1, s);
        exclusive_scan_i64(rk64.as<int64_t>(), rpre.as<int64_t>(), na + 1, s);
    }
    gs.alloc(sizeof(int64_t) * (ng + 1));
    cnt.alloc(sizeof(int64_t) * 5 * (ng + 1));
    cx.alloc(sizeof(int64_t) * 5 * (ng + 1));
    S.K.alloc(sizeof(int32_t) * std::max<int64_t>(ng, 4));
    S.rows.alloc(sizeof(int32_t) * std::max<int64_t>(2 * ng, 4));
    // the scans of the five counts: panel offsets, first columns, item, reduction and slot offsets
    int64_t tot[5] = {0, 0, 0, 0, 0};
    if (ng > 0) {
        bcp_gstart_kernel<<<grid1d_m(na), 256, 0, s>>>(key.as<uint64_t>(), head.as<int64_t>(), gx.as<int64_t>(), na,
                                                        ng, none, gs.as<int64_t>());
        HM_LAUNCH_CHECK();
        bcp_group_kernel<<<grid1d_m(ng + 1), 256, 0, s>>>(key.as<uint64_t>(), gs.as<int64_t>(), rpre.as<int64_t>(),
                                                           ng, nb, S.K.as<int32_t>(), S.rows.as<int32_t>(),
                                                           cnt.as<int64_t>());
        HM_LAUNCH_CHECK();
        for (int q = 0; q < 5; ++q)
            tot[q] = exclusive_scan_i64(cnt.as<int64_t>() + q * (ng + 1), cx.as<int64_t>() + q * (ng + 1), ng + 1, s);
    }
    const int64_t o = tot[0], c = tot[1], ntiles = tot[2], nred = tot[3], nslots = tot[4];
    const int64_t *d_off = cx.as<int64_t>(), *d_col0 = d_off + (ng + 1), *d_toff = d_off + 2 * (ng + 1),
                  *d_roff = d_off + 3 * (ng + 1), *d_soff = d_off + 4 * (ng + 1);
    S.off.alloc(sizeof(int64_t) * (ng + 1));
    S.col0.alloc(sizeof(int64_t) * (ng + 1));
    S.tidx.alloc(std::max<size_t>(sizeof(int32_t) * c, 16));
    S.tiles.alloc(std::max<size_t>(sizeof(int32_t) * BC_ITEM * ntiles, 16));
    S.red.alloc(std::max<size_t>(sizeof(int32_t) * 4 * nred, 16));
    const size_t esz = prec == HM_BF16 ? 2 : 4;
    S.data.alloc(esz * std::max<int64_t>(o, 8));
    HM_CUDA_CHECK(cudaMemsetAsync(S.data.p, 0, esz * std::max<int64_t>(o, 8), s));
    if (ng > 0) {
        HM_CUDA_CHECK(cudaMemcpyAsync(S.off.p, d_off, sizeof(int64_t) * (ng + 1), cudaMemcpyDeviceToDevice, s));
        HM_CUDA_CHECK(cudaMemcpyAsync(S.col0.p, d_col0, sizeof(int64_t) * (ng + 1), cudaMemcpyDeviceToDevice, s));
        fill_i32_kernel<<<grid1d_m(c), 256, 0, s>>>(S.tidx.as<int32_t>(), c, -1);
        HM_LAUNCH_CHECK();
        bcp_block_kernel<<<grid1d_m(na), 256, 0, s>>>(gx.as<int64_t>(), head.as<int64_t>(), gs.as<int64_t>(),
                                                       rpre.as<int64_t>(), id.as<int32_t>(), rk.as<int32_t>(), lofs,
                                                       d_col0, A->t_off.as<int64_t>(), ng, d_bgrp.as<int32_t>(),
                                                       d_bkoff.as<int32_t>(), S.tidx.as<int32_t>());
        HM_LAUNCH_CHECK();
        bcp_items_kernel<<<grid1d_m(ng), 256, 0, s>>>(S.K.as<int32_t>(), S.rows.as<int32_t>(), d_toff, d_roff,
                                                       d_soff, ng, S.tiles.as<int32_t>(), S.red.as<int32_t>());
        HM_LAUNCH_CHECK();
        auto pack = [&](auto *out) {
            using TF = std::remove_pointer_t<decltype(out)>;
            bcp_pack_kernel<TF><<<(unsigned)na, 128, 0, s>>>(
                tr->adm.as<int32_t>(), rk_set, lofs, d_bgrp.as<int32_t>(), d_bkoff.as<int32_t>(), S.off.as<int64_t>(),
                S.K.as<int32_t>(), tr->leaf_begin.as<int32_t>(), tr->n_leaf, tr->lr_colptr.as<int64_t>(),
                tr->lr_collist.as<int32_t>(), A->wp_off.as<int64_t>(), A->wp_K.as<int32_t>(),
                A->wp_koff.as<int32_t>(), A->wp.as<double>(), out);
            HM_LAUNCH_CHECK();
        };
        if (prec == HM_BF16) pack(S.data.as<__nv_bfloat16>());
        else pack(S.data.as<float>());
    }
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
    S.ngroups = ng;
    S.ntiles = ntiles;
    S.nred = nred;
    S.nslots = nslots;
    S.dtype = (int)prec;
}

// The block-column panels of a precision: HM_F32 with BF16 tails gives two
// sets (leading terms FP32, trailing terms BF16), otherwise one set of all
// terms in that precision.
static void build_bcp_sets(const hm_matrix *Ac, hm_dtype prec, cudaStream_t s) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    hm_matrix *A = const_cast<hm_matrix *>(Ac);  // cache owned by the matrix
    if (A->bcp.dtype == (int)prec) return;
    const bool tails = prec == HM_F32 && A->rank32.p && A->ut16.data.p;
    if (!tails) {
        build_bcp(A, A->bcp, prec, A->rank.as<int32_t>(), nullptr, s);
        return;
    }
    const int64_t na = A->tree->n_adm;
    DBuf r16;
    r16.alloc(sizeof(int32_t) * std::max<int64_t>(na, 1));
    if (na > 0) {
        tail_rank_kernel<<<grid1d_m(na), 256, 0, s>>>(A->rank.as<int32_t>(), A->rank32.as<int32_t>(), na,
                                                       r16.as<int32_t>());
        HM_LAUNCH_CHECK();
    }
    A->bcp.dtype = -1;
    build_bcp(A, A->bcp16, HM_BF16, r16.as<int32_t>(), A->rank32.as<int32_t>(), s);
    build_bcp(A, A->bcp, HM_F32, A->rank32.as<int32_t>(), nullptr, s);
}

static int bcp_smem(bool f32) {
    return BP_STAGES * (f32 ? BpStage<float>::BYTES : BpStage<__nv_bfloat16>::BYTES);
}

// Workspace of one 16-column product, in floats: X [n][16] FP32, Y [n][16]
// FP64, then the work of matvec_mrhs_morton: X as BF16 pairs (hi, lo:
// [n][16] each), t as BF16 pairs ([K][16] each) and the partials of the
// projection tiles whose rows were split.  Call mrhs_prepare first.
int64_t mrhs_work_floats(const hm_matrix *A) {
    const int64_t n = A->tree->n, K = std::max<int64_t>(A->total_rank, 1);
    const int64_t P = std::max<int64_t>(std::max(A->bcp.nslots, A->bcp16.nslots), 1);
    return 4 * MR * n + MR * K + P * CM_COLS * MR;  // 48 n + 16 n + 16 K + P
}

void mrhs_prepare(const hm_matrix *A, hm_dtype prec, cudaStream_t s) {
    if ((prec == HM_F32 && A->up32.p) || (prec == HM_BF16 && A->upbf.p)) build_bcp_sets(A, prec, s);
    hm_matrix *Am = const_cast<hm_matrix *>(A);  // cache owned by the matrix
    if (!Am->mrhs_err.p) {
        Am->mrhs_err.alloc(sizeof(int));
        HM_CUDA_CHECK(cudaMemsetAsync(Am->mrhs_err.p, 0, sizeof(int), s));
    }
}

// non-zero when a bounded wait of the tensor-memory row pass gave up since the last call
int mrhs_error(const hm_matrix *A, cudaStream_t s) {
    if (!A->mrhs_err.p) return 0;
    const int e = read_scalar(A->mrhs_err.as<int>(), s);
    if (e) HM_CUDA_CHECK(cudaMemsetAsync(A->mrhs_err.p, 0, sizeof(int), s));
    return e;
}

template <class TF>
void row_mrhs_tc(const hm_matrix *A, const TF *up, const __nv_bfloat16 *Th, const __nv_bfloat16 *Tl,
                 const __nv_bfloat16 *Xh, const __nv_bfloat16 *Xl, double *Y, int *err, cudaStream_t s);



template <int MT, class C> static int row_smem() {
    // the stages, or the per-group sums and the [column][row] output tile
    const int st = C::STAGES * RpStage<MT, float, C>::BYTES, red = C::KG * 16 * MT * MR * 4 + MR * (16 * MT + 1) * 4;
    return st > red ? st : red;
}

// Shapes of the row pass (warps x 16-column groups per slice x stages).  For
// 80-row leaves (MT = 5) measured on the level-8 sphere, FP32 factors, ms per
// product: 4x4x3 7.25, 4x4x2 7.64, 4x4x4 9.98, 8x4x3 7.32, 4x2x5 12.06,
// 4x2x4 9.20, 8x2x4 8.64, 8x2x6 9.91, 8x8x3 9.00, 16x8x2 6.85, 16x8x3 8.32,
// 16x16x2 6.65, 8x8x2 6.42-6.57: wide slices over 8 warps, two stages (111
// KB of shared memory, two CTAs per SM).  The other tile counts keep 4x4x3
// (8x8x2 would hold one CTA per SM for 128-row tiles).
using RpShape5 = RpCfg<8, 8, 2>;
using RpDefault = RpCfg<4, 4, 3>;

// t = W^T X over one set of block-column panels (col_bcp_kernel, then the
// sums of the work items whose rows were split)
template <class TF>
static void col_pass(const BcpSet &S, const __nv_bfloat16 *Xh, const __nv_bfloat16 *Xl, __nv_bfloat16 *Th,
                     __nv_bfloat16 *Tl, float *part, cudaStream_t s) {
    if (S.ntiles == 0) return;
    const bool f32 = sizeof(TF) == 4;
    const int smem = bcp_smem(f32);
    HM_CUDA_CHECK(cudaFuncSetAttribute(col_bcp_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    {
        Trace tc(f32 ? "col_bcp_kernel.f32" : "col_bcp_kernel.bf16", s);
        col_bcp_kernel<TF><<<(unsigned)S.ntiles, CM_THREADS, smem, s>>>(
            S.tiles.as<int32_t>(), S.off.as<int64_t>(), S.K.as<int32_t>(), S.rows.as<int32_t>(), S.col0.as<int64_t>(),
            S.tidx.as<int32_t>(), S.data.as<TF>(), Xh, Xl, Th, Tl, part);
        HM_LAUNCH_CHECK();
    }
    if (S.nred > 0) {
        bcp_reduce_kernel<<<(unsigned)S.nred, 256, 0, s>>>(S.red.as<int32_t>(), S.K.as<int32_t>(),
                                                           S.col0.as<int64_t>(), S.tidx.as<int32_t>(), part, Th, Tl);
        HM_LAUNCH_CHECK();
    }
}

// Y [n][16] FP64 -> the first nr columns of [column][ld] (FP32 / FP64), after the tcgen05 row pass
template <class TO>
__global__ void y_to_cols_kernel(const double *__restrict__ Y, int64_t n, int nr, int64_t ld, TO *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nr; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const int64_t i = e - (int64_t)c * n;
        out[(int64_t)c * ld + i] = (TO)Y[i * MR + c];
    }
}

template <class TF>
static void matvec_mrhs_impl(const hm_matrix *A, const TF *up, const float *X, double *Y, __nv_bfloat16 *Xh,
                             __nv_bfloat16 *Xl, __nv_bfloat16 *Th, __nv_bfloat16 *Tl, float *part, YOut yo,
                             cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t n = tr->n;
    const bool f32 = sizeof(TF) == 4;
    // FP32 factors with BF16 tails: leading terms from the FP32 sets, trailing terms from the BF16 ones
    const bool tails = f32 && A->bcp16.dtype == HM_BF16 && A->ut16.data.p;
    if (X) {  // else the pairs are in place already (matvec_mrhs_cols)
        split_rows_kernel<<<grid1d_m(n * MR), 256, 0, s>>>(X, n * MR, Xh, Xl);
        HM_LAUNCH_CHECK();
    }
    if (tr->n_adm > 0) {
        col_pass<TF>(A->bcp, Xh, Xl, Th, Tl, part, s);
        if (tails) col_pass<__nv_bfloat16>(A->bcp16, Xh, Xl, Th, Tl, part, s);
    }
    const int tiles = (tr->max_leaf + 15) / 16;
    auto launch = [&](auto kern, int smem, int threads) {
        HM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        Trace tr_(f32 ? "row_mrhs_kernel.f32" : "row_mrhs_kernel.bf16", s);
        const TailPanels &U = tails ? A->ut32 : A->ut16;  // ut16: unused (TAIL = false) unless tails
        const TF *u = tails ? reinterpret_cast<const TF *>(A->ut32.data.p) : up;
        kern<<<(unsigned)tr->n_leaf, threads, smem, s>>>(
            tr->leaf_begin.as<int32_t>(), tr->rho_off.as<int64_t>(), tr->rho_K.as<int32_t>(),
            tr->rho_colptr.as<int64_t>(), tr->colidx.as<int32_t>(), A->dense32.as<float>(),
            tails ? U.off.as<int64_t>() : A->up_off.as<int64_t>(), tails ? U.K.as<int32_t>() : A->up_K.as<int32_t>(),
            tails ? U.colptr.as<int64_t>() : A->up_colptr.as<int64_t>(),
            tails ? U.tidx.as<int32_t>() : A->tidx.as<int32_t>(), u, A->ut16.off.as<int64_t>(),
            A->ut16.K.as<int32_t>(), A->ut16.colptr.as<int64_t>(), A->ut16.tidx.as<int32_t>(),
            A->ut16.data.as<__nv_bfloat16>(), Th, Tl, Xh, Xl, Y, yo);
        HM_LAUNCH_CHECK();
    };
    if (A->params.mrhs_tcgen05 && A->mrhs_err.p) {  // the measured tcgen05 / TMEM row pass (mrhs_tc.cu)
        row_mrhs_tc<TF>(A, up, Th, Tl, Xh, Xl, Y, A->mrhs_err.as<int>(), s);
        if (yo.mode == 1)
            y_to_cols_kernel<float><<<grid1d_m(n * yo.nr), 256, 0, s>>>(Y, n, yo.nr, yo.ld, static_cast<float *>(yo.p));
        else if (yo.mode == 2)
            y_to_cols_kernel<double><<<grid1d_m(n * yo.nr), 256, 0, s>>>(Y, n, yo.nr, yo.ld, static_cast<double *>(yo.p));
        HM_LAUNCH_CHECK();
        return;
    }
    using C = RpDefault;
    using C5 = RpShape5;
    if (tails) {
        if constexpr (sizeof(TF) == 4) {
            if (tiles <= 3) launch(row_mrhs_kernel<3, float, C, true>, row_smem<3, C>(), C::THREADS);
            else if (tiles <= 5) launch(row_mrhs_kernel<5, float, C5, true>, row_smem<5, C5>(), C5::THREADS);
            else launch(row_mrhs_kernel<8, float, C, true>, row_smem<8, C>(), C::THREADS);
        }
        return;
    }
    if (tiles <= 3) launch(row_mrhs_kernel<3, TF, C, false>, row_smem<3, C>(), C::THREADS);
    else if (tiles <= 5) launch(row_mrhs_kernel<5, TF, C5, false>, row_smem<5, C5>(), C5::THREADS);
    else launch(row_mrhs_kernel<8, TF, C, false>, row_smem<8, C>(), C::THREADS);
}

// Y (Morton [n][16] FP64) = H X (Morton [n][16] FP32) with the FP32 near field
// and FP32 (prec = HM_F32) or BF16 (HM_BF16) factors.  work: the part of the
// workspace after X and Y (mrhs_work_floats - 48 n floats); mrhs_prepare must
// have run for this precision.  With out (matvec_mrhs_morton_cols) the
// product's first nr columns go straight to out as [column][ld] FP32
// (out_f32) or FP64 instead of Y (Y is then scratch of the tcgen05 form).
static void mrhs_morton(const hm_matrix *A, hm_dtype prec, const float *X, double *Y, float *work, YOut yo,
                        cudaStream_t s) {
    if (!A->dense32.p) fail(HM_EINVAL, "the multi-RHS product needs the FP32 near-field copy");
    if (A->bcp.dtype != (int)prec) fail(HM_EINTERNAL, "multi-RHS panels not prepared for this precision");
    const int64_t n = A->tree->n, K = std::max<int64_t>(A->total_rank, 1);
    __nv_bfloat16 *Xh = reinterpret_cast<__nv_bfloat16 *>(work);
    __nv_bfloat16 *Xl = Xh + MR * n;
    __nv_bfloat16 *Th = Xl + MR * n;
    __nv_bfloat16 *Tl = Th + MR * K;
    float *part = reinterpret_cast<float *>(Tl + MR * K);
    if (prec == HM_F32) {
        if (!A->up32.p) fail(HM_EINVAL, "FP32 copies were not assembled");
        matvec_mrhs_impl<float>(A, A->up32.as<float>(), X, Y, Xh, Xl, Th, Tl, part, yo, s);
    } else if (prec == HM_BF16) {
        if (!A->upbf.p) fail(HM_EINVAL, "BF16 factors were not assembled");
        matvec_mrhs_impl<__nv_bfloat16>(A, A->upbf.as<__nv_bfloat16>(), X, Y, Xh, Xl, Th, Tl, part, yo, s);
    } else {
        fail(HM_EINVAL, "the multi-RHS product runs on the FP32 / BF16 copies");
    }
}

void matvec_mrhs_morton(const hm_matrix *A, hm_dtype prec, const float *X, double *Y, float *work, cudaStream_t s) {
    mrhs_morton(A, prec, X, Y, work, YOut{nullptr, 0, 0, 0}, s);
}

// the product of a block of nr <= 16 vectors x [nr][n] (FP32 when x_f32, else
// FP64; Morton order) into out [nr][n] (FP32 when out_f32, else FP64), the
// BF16 pairs of x made in one pass (no [n][16] FP32 copy); Y: [n][16] FP64
// scratch of the tcgen05 form; work as for matvec_mrhs_morton
void matvec_mrhs_cols(const hm_matrix *A, hm_dtype prec, const void *x, bool x_f32, int nr, double *Y, void *out,
                      bool out_f32, float *work, cudaStream_t s) {
    const int64_t n = A->tree->n;
    __nv_bfloat16 *Xh = reinterpret_cast<__nv_bfloat16 *>(work);
    __nv_bfloat16 *Xl = Xh + MR * n;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + GS_ROWS - 1) / GS_ROWS, 65535));
    if (x_f32)
        gather_split_kernel<float><<<g, 256, 0, s>>>(static_cast<const float *>(x), n, nr, n, Xh, Xl);
    else
        gather_split_kernel<double><<<g, 256, 0, s>>>(static_cast<const double *>(x), n, nr, n, Xh, Xl);
    HM_LAUNCH_CHECK();
    mrhs_morton(A, prec, nullptr, Y, work, YOut{out, n, nr, out_f32 ? 1 : 2}, s);
}

// y = alpha H x + beta y for up to 16 right-hand sides [nrhs][n] (original
// order), through the tensor-core product.  Stream-ordered scratch.
void matvec_mrhs(const hm_matrix *A, hm_dtype prec, int nrhs, const double *x, double *y, double alpha, double beta,
                 cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t n = tr->n;
    mrhs_prepare(A, prec, s);
    for (int r0 = 0; r0 < nrhs; r0 += MR) {
        const int nr = std::min(MR, nrhs - r0);
        SBuf buf;
        buf.alloc(sizeof(float) * mrhs_work_floats(A), s);
        float *X = buf.as<float>();
        double *Y = reinterpret_cast<double *>(X + MR * n);  // [n][16] doubles = 2 * 16 * n floats
        float *work = X + 3 * MR * n;
        mrhs_gather_kernel<<<grid1d_m(n * MR), 256, 0, s>>>(x + (int64_t)r0 * n, n, nr, tr->perm.as<int32_t>(), X);
        HM_LAUNCH_CHECK();
        matvec_mrhs_morton(A, prec, X, Y, work, s);
        mrhs_scatter_kernel<<<grid1d_m(n * nr), 256, 0, s>>>(Y, n, nr, tr->perm.as<int32_t>(), alpha, beta,
                                                             y + (int64_t)r0 * n);
        HM_LAUNCH_CHECK();
    }
}

}  // namespace hm
