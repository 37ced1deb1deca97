// mrhs.cu -- H-matrix product with 16 right-hand sides at once on the tensor
// cores (the multi-RHS form of the H-matvec of Sec. 2.3).
//
// With one right-hand side the product reads every stored entry for one
// multiply-add (HBM-bound, CUDA cores).  With 16 it is 16 multiply-adds per
// entry: 32 flops per 4-byte near-field entry and per 2-byte BF16 factor
// entry, above what the FP32 CUDA cores deliver at HBM speed, so the three
// passes of the product become small GEMMs on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation):
//   col_mrhs_kernel : P_kappa (16 x K_kappa) = X_kappa^T W~_kappa per leaf
//                     column cluster (A = X^T from shared memory, B = panel
//                     tile staged by cp.async and read with ldmatrix.trans);
//   tsum_mrhs_kernel: t_b = sum of the partials over the clusters of b;
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
// Layout: X [n][16] FP32 and Y [n][16] FP64 in Morton order, the partials
// [P][16], t [K][16] (rows = panel columns / t entries, 16 right-hand sides
// contiguous).
#include <cuda_bf16.h>

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

// ---------------------------------------------------------------------------
// col_mrhs_kernel: partials of X_kappa^T W~_kappa, one CTA per leaf column
// cluster.  The W panel (|kappa| x Kw, row-major, BF16 or FP32) is walked in
// tiles of 64 columns; each warp owns 8 columns of a tile.
// ---------------------------------------------------------------------------
constexpr int CM_THREADS = 256;
constexpr int CM_COLS = 64;                 // panel columns per tile
constexpr int CM_TSTRIDE = CM_COLS + 8;     // bf16 per tile row in shared memory (16-byte aligned rows)

template <class TF> struct ColTile;
// BF16 panels: the tile goes to shared memory as is (cp.async), one operand
template <> struct ColTile<__nv_bfloat16> {
    static constexpr int NSPLIT = 1;
};
// FP32 panels: staged as FP32, then split into BF16 hi / lo tiles
template <> struct ColTile<float> {
    static constexpr int NSPLIT = 2;
};

template <class TF>
__global__ void __launch_bounds__(CM_THREADS) col_mrhs_kernel(const int32_t *__restrict__ leaf_begin,
                                                              const int64_t *__restrict__ wp_off,
                                                              const int32_t *__restrict__ wp_K,
                                                              const int64_t *__restrict__ wp_colptr,
                                                              const TF *__restrict__ wp, const float *__restrict__ X,
                                                              float *__restrict__ P) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int64_t kap = blockIdx.x;
    const int32_t c0 = leaf_begin[kap], mc = leaf_begin[kap + 1] - c0;
    const int kpad = (mc + 15) & ~15;
    const int Kw = wp_K[kap];
    const TF *W = wp + wp_off[kap];
    float *out = P + wp_colptr[kap] * MR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    // shared: X^T hi / lo [16][kpad + 8] bf16, then the tile(s) [kpad][CM_TSTRIDE] bf16 (x NSPLIT), then for
    // FP32 panels the FP32 staging tile [kpad][CM_COLS]
    const int xs = kpad + 8;
    __nv_bfloat16 *sXh = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *sXl = sXh + MR * xs;
    __nv_bfloat16 *sT = sXl + MR * xs;
    float *sF = reinterpret_cast<float *>(sT + ColTile<TF>::NSPLIT * kpad * CM_TSTRIDE);
    for (int e = threadIdx.x; e < MR * kpad; e += CM_THREADS) {
        const int r = e / kpad, k = e - (e / kpad) * kpad;
        float h = 0.0f, l = 0.0f;
        if (k < mc) split_bf16(X[(int64_t)(c0 + k) * MR + r], h, l);
        sXh[r * xs + k] = __float2bfloat16_rn(h);
        sXl[r * xs + k] = __float2bfloat16_rn(l);
    }
    __syncthreads();
    const int nk = kpad / 16;
    for (int n0 = 0; n0 < Kw; n0 += CM_COLS) {
        // stage the tile rows [0, kpad) x columns [n0, n0 + 64); rows >= mc and columns >= Kw read as 0
        if constexpr (sizeof(TF) == 2) {
            for (int e = threadIdx.x; e < kpad * (CM_COLS / 8); e += CM_THREADS) {
                const int k = e / (CM_COLS / 8), v = e - (e / (CM_COLS / 8)) * (CM_COLS / 8);
                const int col = n0 + 8 * v;
                const bool ok = k < mc && col < Kw;
                cp_async16(sT + k * CM_TSTRIDE + 8 * v, ok ? (const void *)(W + (int64_t)k * Kw + col) : (const void *)W,
                           ok);
            }
            cp_async_commit();
            cp_async_wait<0>();
        } else {
            for (int e = threadIdx.x; e < kpad * (CM_COLS / 4); e += CM_THREADS) {
                const int k = e / (CM_COLS / 4), v = e - (e / (CM_COLS / 4)) * (CM_COLS / 4);
                const int col = n0 + 4 * v;
                const bool ok = k < mc && col < Kw;
                cp_async16(sF + k * CM_COLS + 4 * v, ok ? (const void *)(W + (int64_t)k * Kw + col) : (const void *)W,
                           ok);
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            for (int e = threadIdx.x; e < kpad * CM_COLS; e += CM_THREADS) {
                const int k = e / CM_COLS, c = e - (e / CM_COLS) * CM_COLS;
                float h, l;
                split_bf16(sF[e], h, l);
                sT[k * CM_TSTRIDE + c] = __float2bfloat16_rn(h);
                sT[kpad * CM_TSTRIDE + k * CM_TSTRIDE + c] = __float2bfloat16_rn(l);
            }
        }
        __syncthreads();
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int ks = 0; ks < nk; ++ks) {
            // A = X^T (16 rhs x 16 k): rows g, g + 8; k pairs (2t, 2t+1), (2t+8, 2t+9)
            const int kb = ks * 16;
            const uint32_t ah0 = *reinterpret_cast<const uint32_t *>(sXh + g * xs + kb + 2 * t);
            const uint32_t ah1 = *reinterpret_cast<const uint32_t *>(sXh + (g + 8) * xs + kb + 2 * t);
            const uint32_t ah2 = *reinterpret_cast<const uint32_t *>(sXh + g * xs + kb + 2 * t + 8);
            const uint32_t ah3 = *reinterpret_cast<const uint32_t *>(sXh + (g + 8) * xs + kb + 2 * t + 8);
            const uint32_t al0 = *reinterpret_cast<const uint32_t *>(sXl + g * xs + kb + 2 * t);
            const uint32_t al1 = *reinterpret_cast<const uint32_t *>(sXl + (g + 8) * xs + kb + 2 * t);
            const uint32_t al2 = *reinterpret_cast<const uint32_t *>(sXl + g * xs + kb + 2 * t + 8);
            const uint32_t al3 = *reinterpret_cast<const uint32_t *>(sXl + (g + 8) * xs + kb + 2 * t + 8);
            // B = tile rows kb..kb+15, columns 8 warp .. +7: ldmatrix.trans, row addresses from lanes 0..15
            uint32_t b0, b1;
            ldmatrix_x2_trans(b0, b1, sT + (kb + (lane & 15)) * CM_TSTRIDE + 8 * warp);
            mma_bf16(d, ah0, ah1, ah2, ah3, b0, b1);
            mma_bf16(d, al0, al1, al2, al3, b0, b1);
            if constexpr (ColTile<TF>::NSPLIT == 2) {
                uint32_t e0, e1;
                ldmatrix_x2_trans(e0, e1, sT + kpad * CM_TSTRIDE + (kb + (lane & 15)) * CM_TSTRIDE + 8 * warp);
                mma_bf16(d, ah0, ah1, ah2, ah3, e0, e1);
            }
        }
        // D (16 rhs x 8 columns): rows g, g + 8, columns 2t, 2t + 1 of this warp's 8
        const int col = n0 + 8 * warp + 2 * t;
        if (col < Kw) {
            out[(int64_t)col * MR + g] = d[0];
            out[(int64_t)col * MR + g + 8] = d[2];
        }
        if (col + 1 < Kw) {
            out[(int64_t)(col + 1) * MR + g] = d[1];
            out[(int64_t)(col + 1) * MR + g + 8] = d[3];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// tsum_mrhs_kernel: t_b(l, :) = sum over the clusters of b of the partials,
// in increasing cluster order.  Two t entries per warp (16 lanes each, one
// lane per right-hand side); the block of an entry is found from the table
// of the block holding every 32nd entry.
// ---------------------------------------------------------------------------
__global__ void tsum_mrhs_kernel(int64_t na, int64_t nt, const int32_t *__restrict__ b0tab,
                                 const int64_t *__restrict__ t_off, const int64_t *__restrict__ bptr,
                                 const int64_t *__restrict__ pofs, const float *__restrict__ P,
                                 float *__restrict__ T) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q0 = tid; q0 < nt * MR; q0 += nthreads) {
        const int64_t e = q0 / MR;
        const int r = (int)(q0 - e * MR);
        int64_t b = b0tab[e / 32];
        while (b + 1 < na && t_off[b + 1] <= e) ++b;
        const int l = (int)(e - t_off[b]);
        float acc = 0.0f;
        for (int64_t q = bptr[b]; q < bptr[b + 1]; ++q) acc += P[(pofs[q] + l) * MR + r];
        T[e * MR + r] = acc;
    }
}

// ---------------------------------------------------------------------------
// row_mrhs_kernel: Y_rho = P_rho X(colidx) + U~_rho T(tidx), one CTA per leaf
// row cluster, MT tiles of 16 rows per pass.  Per staged chunk of 256 panel
// columns every warp takes 32 of them: its A fragments come straight from the
// panel rows with one 16-byte load per row and 16 (FP32) or 32 (BF16)
// columns, the k order inside a 16-k step permuted consistently in A and B
// (B read from the staged chunk at the same physical columns).
// ---------------------------------------------------------------------------
constexpr int RM_THREADS = 256;
constexpr int RM_WARPS = RM_THREADS / 32;
constexpr int RM_CHUNK = 256;           // panel columns staged per pass
constexpr int RM_BSTRIDE = RM_CHUNK + 16;  // bf16 per right-hand side row in shared memory

// FP32 panel: A fragment of rows (row g, row g + 8) for physical columns
// 4t .. 4t + 3 of a 16-column group, split hi / lo
__device__ __forceinline__ void a_frag_f32(const float *r0, const float *r1, bool v0, bool v1, uint32_t (&ah)[4],
                                           uint32_t (&al)[4]) {
    float4 p = v0 ? __ldg(reinterpret_cast<const float4 *>(r0)) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 q = v1 ? __ldg(reinterpret_cast<const float4 *>(r1)) : make_float4(0.f, 0.f, 0.f, 0.f);
    float h[8], l[8];
    split_bf16(p.x, h[0], l[0]);
    split_bf16(p.y, h[1], l[1]);
    split_bf16(p.z, h[2], l[2]);
    split_bf16(p.w, h[3], l[3]);
    split_bf16(q.x, h[4], l[4]);
    split_bf16(q.y, h[5], l[5]);
    split_bf16(q.z, h[6], l[6]);
    split_bf16(q.w, h[7], l[7]);
    // logical (2t, 2t+1) <- physical (4t, 4t+1); (2t+8, 2t+9) <- (4t+2, 4t+3)
    ah[0] = pack_bf16(h[0], h[1]);
    ah[1] = pack_bf16(h[4], h[5]);
    ah[2] = pack_bf16(h[2], h[3]);
    ah[3] = pack_bf16(h[6], h[7]);
    al[0] = pack_bf16(l[0], l[1]);
    al[1] = pack_bf16(l[4], l[5]);
    al[2] = pack_bf16(l[2], l[3]);
    al[3] = pack_bf16(l[6], l[7]);
}

template <class TP> struct RowPanel;
// FP32 near field / factors: 4 columns per 16-byte load, three products
template <> struct RowPanel<float> {
    static constexpr int PER_LOAD = 4;
};
// BF16 factors: 8 columns per 16-byte load, exact operand, two products
template <> struct RowPanel<__nv_bfloat16> {
    static constexpr int PER_LOAD = 8;
};

template <int MT, class TP>
__device__ __forceinline__ void row_mrhs_panel(const TP *__restrict__ Pn, int K, const int32_t *__restrict__ idx,
                                               const float *__restrict__ Z, int mr, int r0t,
                                               __nv_bfloat16 *sBh, __nv_bfloat16 *sBl, float (&acc)[MT][2][4]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    for (int c0 = 0; c0 < K; c0 += RM_CHUNK) {
        __syncthreads();
        // gathered rows of Z for the chunk's columns, split into BF16 hi / lo, [rhs][column]
        for (int c = threadIdx.x; c < RM_CHUNK; c += RM_THREADS) {
            const int col = c0 + c;
            float z[MR];
            if (col < K) {
                const float4 *zr = reinterpret_cast<const float4 *>(Z + (int64_t)idx[col] * MR);
#pragma unroll
                for (int v = 0; v < MR / 4; ++v) {
                    const float4 q = __ldg(zr + v);
                    z[4 * v] = q.x;
                    z[4 * v + 1] = q.y;
                    z[4 * v + 2] = q.z;
                    z[4 * v + 3] = q.w;
                }
            } else {
#pragma unroll
                for (int r = 0; r < MR; ++r) z[r] = 0.0f;
            }
#pragma unroll
            for (int r = 0; r < MR; ++r) {
                float h, l;
                split_bf16(z[r], h, l);
                sBh[r * RM_BSTRIDE + c] = __float2bfloat16_rn(h);
                sBl[r * RM_BSTRIDE + c] = __float2bfloat16_rn(l);
            }
        }
        __syncthreads();
        // this warp's 32 columns of the chunk
        const int wc = warp * 32;
        if (c0 + wc >= K) continue;
        if constexpr (RowPanel<TP>::PER_LOAD == 4) {
#pragma unroll
            for (int grp = 0; grp < 2; ++grp) {
                const int pc = wc + 16 * grp + 4 * t;  // physical column of this thread's 4 values (chunk-relative)
                const bool colok = c0 + pc < K;
                // B fragments at the same physical columns: rhs g (n-tile 0) and g + 8 (n-tile 1)
                uint32_t bh[2][2], bl[2][2];
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const uint2 vh = *reinterpret_cast<const uint2 *>(sBh + (g + 8 * nt) * RM_BSTRIDE + pc);
                    const uint2 vl = *reinterpret_cast<const uint2 *>(sBl + (g + 8 * nt) * RM_BSTRIDE + pc);
                    bh[nt][0] = vh.x;
                    bh[nt][1] = vh.y;
                    bl[nt][0] = vl.x;
                    bl[nt][1] = vl.y;
                }
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    const int ra = r0t + 16 * mt + g, rb = ra + 8;
                    uint32_t ah[4], al[4];
                    a_frag_f32(reinterpret_cast<const float *>(Pn) + (int64_t)(ra < mr ? ra : 0) * K + c0 + pc,
                               reinterpret_cast<const float *>(Pn) + (int64_t)(rb < mr ? rb : 0) * K + c0 + pc,
                               colok && ra < mr, colok && rb < mr, ah, al);
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        mma_bf16(acc[mt][nt], ah[0], ah[1], ah[2], ah[3], bh[nt][0], bh[nt][1]);
                        mma_bf16(acc[mt][nt], ah[0], ah[1], ah[2], ah[3], bl[nt][0], bl[nt][1]);
                        mma_bf16(acc[mt][nt], al[0], al[1], al[2], al[3], bh[nt][0], bh[nt][1]);
                    }
                }
            }
        } else {
            const int pc = wc + 8 * t;  // physical columns pc .. pc + 7 (chunk-relative)
            const bool colok = c0 + pc < K;
            // two k16 products: physical (pc .. pc+3) and (pc+4 .. pc+7)
            uint32_t bh[2][2][2], bl[2][2][2];  // [half][n-tile][reg]
#pragma unroll
            for (int hf = 0; hf < 2; ++hf)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const uint2 vh = *reinterpret_cast<const uint2 *>(sBh + (g + 8 * nt) * RM_BSTRIDE + pc + 4 * hf);
                    const uint2 vl = *reinterpret_cast<const uint2 *>(sBl + (g + 8 * nt) * RM_BSTRIDE + pc + 4 * hf);
                    bh[hf][nt][0] = vh.x;
                    bh[hf][nt][1] = vh.y;
                    bl[hf][nt][0] = vl.x;
                    bl[hf][nt][1] = vl.y;
                }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const int ra = r0t + 16 * mt + g, rb = ra + 8;
                const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
                const uint4 p = (colok && ra < mr)
                                    ? __ldg(reinterpret_cast<const uint4 *>(Pn + (int64_t)ra * K + c0 + pc))
                                    : zero;
                const uint4 q = (colok && rb < mr)
                                    ? __ldg(reinterpret_cast<const uint4 *>(Pn + (int64_t)rb * K + c0 + pc))
                                    : zero;
                // half 0: logical (2t,2t+1) <- (pc, pc+1) = p.x, (2t+8, 2t+9) <- (pc+2, pc+3) = p.y
                // half 1: p.z, p.w
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    mma_bf16(acc[mt][nt], p.x, q.x, p.y, q.y, bh[0][nt][0], bh[0][nt][1]);
                    mma_bf16(acc[mt][nt], p.x, q.x, p.y, q.y, bl[0][nt][0], bl[0][nt][1]);
                    mma_bf16(acc[mt][nt], p.z, q.z, p.w, q.w, bh[1][nt][0], bh[1][nt][1]);
                    mma_bf16(acc[mt][nt], p.z, q.z, p.w, q.w, bl[1][nt][0], bl[1][nt][1]);
                }
            }
        }
    }
}

template <int MT, class TF>
__global__ void __launch_bounds__(RM_THREADS) row_mrhs_kernel(
    const int32_t *__restrict__ leaf_begin, const int64_t *__restrict__ rho_off, const int32_t *__restrict__ rho_K,
    const int64_t *__restrict__ rho_colptr, const int32_t *__restrict__ colidx, const float *__restrict__ dense,
    const int64_t *__restrict__ up_off, const int32_t *__restrict__ up_K, const int64_t *__restrict__ up_colptr,
    const int32_t *__restrict__ tidx, const TF *__restrict__ up, const float *__restrict__ T,
    const float *__restrict__ X, double *__restrict__ Y) {
    extern __shared__ __align__(16) unsigned char sm[];
    __nv_bfloat16 *sBh = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *sBl = sBh + MR * RM_BSTRIDE;
    float *sRed = reinterpret_cast<float *>(sBl + MR * RM_BSTRIDE);  // [warps][16 * MT rows][16]
    const int64_t rho = blockIdx.x;
    const int32_t r0 = leaf_begin[rho], mr = leaf_begin[rho + 1] - r0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    for (int r0t = 0; r0t < mr; r0t += 16 * MT) {
        float acc[MT][2][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
        row_mrhs_panel<MT, float>(dense + rho_off[rho], rho_K[rho], colidx + rho_colptr[rho], X, mr, r0t, sBh, sBl,
                                  acc);
        row_mrhs_panel<MT, TF>(up + up_off[rho], up_K[rho], tidx + up_colptr[rho], T, mr, r0t, sBh, sBl, acc);
        // per-warp partial sums -> shared memory -> fixed-order sum over warps
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                float *base = sRed + (int64_t)warp * (16 * MT) * MR;
                const int ra = 16 * mt + g, col = 8 * nt + 2 * t;
                base[ra * MR + col] = acc[mt][nt][0];
                base[ra * MR + col + 1] = acc[mt][nt][1];
                base[(ra + 8) * MR + col] = acc[mt][nt][2];
                base[(ra + 8) * MR + col + 1] = acc[mt][nt][3];
            }
        __syncthreads();
        const int rows = min(16 * MT, mr - r0t);
        for (int e = threadIdx.x; e < rows * MR; e += RM_THREADS) {
            float s = 0.0f;
            for (int w = 0; w < RM_WARPS; ++w) s += sRed[(int64_t)w * (16 * MT) * MR + e];
            Y[(int64_t)(r0 + r0t) * MR + e] = (double)s;
        }
        __syncthreads();
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

int64_t mrhs_work_floats(const hm_matrix *A) {
    const int64_t n = A->tree->n;
    return MR * (n + std::max<int64_t>(A->n_partials, 1) + std::max<int64_t>(A->total_rank, 1)) + 2 * MR * n;
}

static int col_smem(int max_leaf, bool f32) {
    const int kpad = (max_leaf + 15) & ~15;
    int b = 2 * MR * (kpad + 8) * 2 + (f32 ? 2 : 1) * kpad * CM_TSTRIDE * 2;
    if (f32) b += kpad * CM_COLS * 4;
    return (b + 15) & ~15;
}

template <int MT> static int row_smem() { return 2 * MR * RM_BSTRIDE * 2 + RM_WARPS * 16 * MT * MR * 4; }

template <class TF>
static void matvec_mrhs_impl(const hm_matrix *A, const TF *up, const TF *wp, const float *X, float *P, float *T,
                             double *Y, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const bool f32 = sizeof(TF) == 4;
    if (tr->n_adm > 0) {
        const int smem = col_smem(tr->max_leaf, f32);
        HM_CUDA_CHECK(cudaFuncSetAttribute(col_mrhs_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        Trace tc(f32 ? "col_mrhs_kernel.f32" : "col_mrhs_kernel.bf16", s);
        col_mrhs_kernel<TF><<<(unsigned)tr->n_leaf, CM_THREADS, smem, s>>>(
            tr->leaf_begin.as<int32_t>(), A->wp_off.as<int64_t>(), A->wp_K.as<int32_t>(), A->wp_colptr.as<int64_t>(),
            wp, X, P);
        HM_LAUNCH_CHECK();
    }
    if (tr->n_adm > 0) {
        Trace tt("tsum_mrhs_kernel", s);
        tsum_mrhs_kernel<<<grid1d_m(A->total_rank * MR), 256, 0, s>>>(
            tr->n_adm, A->total_rank, A->tsum_b0.as<int32_t>(), A->t_off.as<int64_t>(), tr->lr_bcolptr.as<int64_t>(),
            A->pofs.as<int64_t>(), P, T);
        HM_LAUNCH_CHECK();
    }
    const int tiles = (tr->max_leaf + 15) / 16;
    auto launch = [&](auto kern, int smem) {
        HM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        Trace tr_(f32 ? "row_mrhs_kernel.f32" : "row_mrhs_kernel.bf16", s);
        kern<<<(unsigned)tr->n_leaf, RM_THREADS, smem, s>>>(
            tr->leaf_begin.as<int32_t>(), tr->rho_off.as<int64_t>(), tr->rho_K.as<int32_t>(),
            tr->rho_colptr.as<int64_t>(), tr->colidx.as<int32_t>(), A->dense32.as<float>(), A->up_off.as<int64_t>(),
            A->up_K.as<int32_t>(), A->up_colptr.as<int64_t>(), A->tidx.as<int32_t>(), up, T, X, Y);
        HM_LAUNCH_CHECK();
    };
    if (tiles <= 3) launch(row_mrhs_kernel<3, TF>, row_smem<3>());
    else if (tiles <= 5) launch(row_mrhs_kernel<5, TF>, row_smem<5>());
    else launch(row_mrhs_kernel<4, TF>, row_smem<4>());
}

// Y (Morton [n][16] FP64) = H X (Morton [n][16] FP32) with the FP32 near field
// and FP32 (prec = HM_F32) or BF16 (HM_BF16) factors.  work: mrhs_work_floats.
void matvec_mrhs_morton(const hm_matrix *A, hm_dtype prec, const float *X, double *Y, float *work, cudaStream_t s) {
    if (!A->dense32.p) fail(HM_EINVAL, "the multi-RHS product needs the FP32 near-field copy");
    const int64_t n = A->tree->n;
    float *P = work;
    float *T = P + MR * std::max<int64_t>(A->n_partials, 1);
    (void)n;
    if (prec == HM_F32) {
        if (!A->up32.p) fail(HM_EINVAL, "FP32 copies were not assembled");
        matvec_mrhs_impl<float>(A, A->up32.as<float>(), A->wp32.as<float>(), X, P, T, Y, s);
    } else if (prec == HM_BF16) {
        if (!A->upbf.p) fail(HM_EINVAL, "BF16 factors were not assembled");
        matvec_mrhs_impl<__nv_bfloat16>(A, A->upbf.as<__nv_bfloat16>(), A->wpbf.as<__nv_bfloat16>(), X, P, T, Y, s);
    } else {
        fail(HM_EINVAL, "the multi-RHS product runs on the FP32 / BF16 copies");
    }
}

// y = alpha H x + beta y for up to 16 right-hand sides [nrhs][n] (original
// order), through the tensor-core product.  Stream-ordered scratch.
void matvec_mrhs(const hm_matrix *A, hm_dtype prec, int nrhs, const double *x, double *y, double alpha, double beta,
                 cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t n = tr->n;
    for (int r0 = 0; r0 < nrhs; r0 += MR) {
        const int nr = std::min(MR, nrhs - r0);
        SBuf buf;
        const int64_t nf = mrhs_work_floats(A);
        buf.alloc(sizeof(float) * nf, s);
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
