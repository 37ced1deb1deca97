// mrhs_df.cu -- the product of the FP64 master with up to 16 right-hand
// sides (the H-matvec of Sec. 2.3) in double-float arithmetic, for the FP64
// residuals of the iterative refinement and hm_matvec_block(HM_F64).
//
// GB300 runs FP64 FMAs at 2 per SM and clock, FP32 FMAs at 128: the FP64
// products of the refinement (one per system, each reading the whole FP64
// master) are bound by the FP64 pipe.  Here every stored FP64 entry w is read
// once per 16 right-hand sides and split into an unevaluated pair of floats,
// w = h + l (h: w truncated to 24 significant bits, l: the rest rounded to
// 24), by integer operations (no FP64 instruction); x is split the same way
// (by FP64 conversions, n values).  Each term is accumulated into a pair
// (s, c) of floats with an error-free product (TwoProduct: p + e = h_w h_x
// exactly, by one FMA) and an error-free sum (TwoSum: s + p = t + sigma
// exactly), the cross terms h_w l_x + l_w h_x and the two errors going to c:
// the compensated dot product of Ogita, Rump and Oishi (2005, "Accurate sum
// and dot product", Algorithm 5.3, Dot2) with double-float operands.  Its
// result carries about 2^-47 relative error per term plus the rounding of
// the compensation (n u^2 |H||x| at worst for n terms, u = 2^-24, about
// sqrt(n) u^2 typically: ~1e-13 of a row sum of |H||x| at worst, a few 1e-15
// in norm), against 2^-53 per term of the FP64 product; two orders below the
// 1e-12 residuals the refinement stops at.
//
// The three passes of the FP64 product, each with 16 right-hand sides:
//   col_df_kernel : per leaf column cluster kappa, the partials x_kappa^T W
//                   of its column panel (one thread per panel column, all 16
//                   right-hand sides in registers, x_kappa staged in shared
//                   memory);
//   tsum_df_kernel: t_b = sum of b's partials in increasing cluster order;
//   row_df_kernel : per leaf row cluster, the near-field panel times the
//                   gathered x and the U panel times the gathered t (panel
//                   chunks staged by cp.async, the K range shared by KS
//                   thread groups, combined in a fixed order at the end).
// The products use __fmul_rn / __fadd_rn / __fsub_rn so that no FMA
// contraction changes the error-free transformations.
#include <algorithm>

#include "hm_internal.cuh"

namespace hm {
namespace df {

constexpr int MR = 16;

// w = h + l: h is w truncated to 24 significant bits, l = w - h rounded to
// 24 bits (|w - h - l| <= 2^-47 |w|), from the bits of w: for 2^-74 <= |w| <
// 2^128 the exponent and the top 23 fraction bits of w make h, the low 29
// fraction bits (an integer m) make l = m 2^(e - 52) with e the unbiased
// exponent of w.  |w| < 2^-126 (zeros included) gives (0, 0); the remaining
// ranges, which BEM entries do not reach, use FP64 conversions.
__device__ __forceinline__ void split(double w, float &h, float &l) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(w);
    const uint32_t hi32 = (uint32_t)(b >> 32), lo32 = (uint32_t)b;
    const uint32_t mag = hi32 & 0x7fffffffu, sgn = hi32 & 0x80000000u;
    if (mag >= 0x3b500000u && mag < 0x47f00000u) {  // biased exponent in [949, 1151)
        h = __uint_as_float(sgn | ((mag - 0x38000000u) << 3) | (lo32 >> 29));
        const float m = __uint2float_rn(lo32 & 0x1fffffffu);
        const float sc = __uint_as_float((uint32_t)((int)(mag >> 20) - 948) << 23);  // 2^(e - 52)
        l = __uint_as_float(__float_as_uint(__fmul_rn(m, sc)) | sgn);
    } else if (mag < 0x38100000u) {
        h = 0.0f;
        l = 0.0f;
    } else {
        h = __double2float_rz(w);
        l = __double2float_rn(w - (double)h);
    }
}

// (s, c) += (ah + al)(xh + xl): TwoProduct and TwoSum; the two errors and
// the cross terms are summed first and reach c in one rounding per term (the
// rounding errors of c itself are what bound the result: ~sqrt(n) u |c|)
__device__ __forceinline__ void dfma(float &s, float &c, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    const float e = __fmaf_rn(ah, xh, -p);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float sg = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fmaf_rn(al, xh, __fmaf_rn(ah, xl, __fadd_rn(e, sg))));
}

// (s, c) += (s2, c2)
__device__ __forceinline__ void dadd(float &s, float &c, float s2, float c2) {
    const float t = __fadd_rn(s, s2);
    const float bp = __fsub_rn(t, s);
    const float sg = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, sg));
}

// (s, c) -> (h, l) with h = fl(s + c), h + l = s + c exactly (TwoSum)
__device__ __forceinline__ void norm2(float s, float c, float &h, float &l) {
    h = __fadd_rn(s, c);
    const float bp = __fsub_rn(h, s);
    l = __fadd_rn(__fsub_rn(s, __fsub_rn(h, bp)), __fsub_rn(c, bp));
}

// X{h,l}[m][r] = x_r at Morton position m (x is [nr][n], original order when
// perm is given), split into floats; zeros for r >= nr
__global__ void split_x_kernel(const double *__restrict__ x, int64_t n, int nr, const int32_t *__restrict__ perm,
                               float *__restrict__ Xh, float *__restrict__ Xl) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * MR; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / MR;
        const int r = (int)(e - m * MR);
        const double v = r < nr ? x[(int64_t)r * n + (perm ? perm[m] : m)] : 0.0;
        const float h = __double2float_rn(v);
        Xh[e] = h;
        Xl[e] = __double2float_rn(v - (double)h);
    }
}

// ---------------------------------------------------------------------------
// column pass: P[wp_colptr[kappa] + v][r] = sum_j W_kappa[j][v] x_r[c0 + j]
// ---------------------------------------------------------------------------
constexpr int CD_THREADS = 256;

__device__ __forceinline__ void col_step(double w, const float4 *sx, float (&s)[MR], float (&c)[MR]) {
    float ah, al;
    split(w, ah, al);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const float4 xh = sx[g], xl = sx[4 + g];
        dfma(s[4 * g], c[4 * g], ah, al, xh.x, xl.x);
        dfma(s[4 * g + 1], c[4 * g + 1], ah, al, xh.y, xl.y);
        dfma(s[4 * g + 2], c[4 * g + 2], ah, al, xh.z, xl.z);
        dfma(s[4 * g + 3], c[4 * g + 3], ah, al, xh.w, xl.w);
    }
}

__global__ void __launch_bounds__(CD_THREADS) col_df_kernel(const int32_t *__restrict__ leaf_begin,
                                                            const int64_t *__restrict__ wp_off,
                                                            const int32_t *__restrict__ wp_K,
                                                            const int64_t *__restrict__ wp_colptr,
                                                            const double *__restrict__ wp, const float *__restrict__ Xh,
                                                            const float *__restrict__ Xl, float2 *__restrict__ P,
                                                            const int32_t *__restrict__ order) {
    __shared__ float4 sx[MAX_LEAF * 8];  // row j of x_kappa: hi [16] then lo [16]
    const int64_t kap = order ? order[blockIdx.x] : blockIdx.x;
    const int32_t c0 = leaf_begin[kap], mc = leaf_begin[kap + 1] - c0;
    const float4 *xh4 = reinterpret_cast<const float4 *>(Xh), *xl4 = reinterpret_cast<const float4 *>(Xl);
    for (int e = threadIdx.x; e < mc * 8; e += CD_THREADS) {
        const int j = e >> 3, q = e & 7;
        sx[e] = q < 4 ? xh4[(int64_t)(c0 + j) * 4 + q] : xl4[(int64_t)(c0 + j) * 4 + q - 4];
    }
    __syncthreads();
    const int Kw = wp_K[kap];
    const double *W = wp + wp_off[kap];
    float4 *out = reinterpret_cast<float4 *>(P + wp_colptr[kap] * MR);
    for (int v = threadIdx.x; v < Kw; v += CD_THREADS) {
        float s[MR], c[MR];
#pragma unroll
        for (int r = 0; r < MR; ++r) s[r] = c[r] = 0.0f;
        const double *col = W + v;
        int j = 0;
        for (; j + 3 < mc; j += 4) {  // four loads in flight
            const double w0 = __ldg(col + (int64_t)j * Kw), w1 = __ldg(col + (int64_t)(j + 1) * Kw);
            const double w2 = __ldg(col + (int64_t)(j + 2) * Kw), w3 = __ldg(col + (int64_t)(j + 3) * Kw);
            col_step(w0, sx + j * 8, s, c);
            col_step(w1, sx + (j + 1) * 8, s, c);
            col_step(w2, sx + (j + 2) * 8, s, c);
            col_step(w3, sx + (j + 3) * 8, s, c);
        }
        for (; j < mc; ++j) col_step(__ldg(col + (int64_t)j * Kw), sx + j * 8, s, c);
#pragma unroll
        for (int r = 0; r < MR; r += 2) out[(int64_t)v * 8 + r / 2] = make_float4(s[r], c[r], s[r + 1], c[r + 1]);
    }
}

// ---------------------------------------------------------------------------
// t_b(l) = sum over the column clusters of sigma_b of the partials, in
// increasing cluster order: one lane per entry of t (all 16 right-hand
// sides), 32 consecutive entries per warp; the entry's block is found from
// b0[c] (the block holding entry 32 c) by a search over the next 32 blocks'
// offsets, or over t_off beyond them.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tsum_df_kernel(int64_t na, int64_t nt, const int32_t *__restrict__ b0tab,
                                                      const int64_t *__restrict__ t_off,
                                                      const int64_t *__restrict__ bcolptr,
                                                      const int64_t *__restrict__ pofs, const float2 *__restrict__ P,
                                                      float *__restrict__ Th, float *__restrict__ Tl) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunk = (nt + 31) / 32;
    for (int64_t ch = w0; ch < nchunk; ch += nw) {
        const int64_t b0 = b0tab[ch];
        const int64_t bl = min(b0 + lane, na);
        const int64_t to = t_off[bl];  // t_off has na + 1 entries
        const int64_t e = ch * 32 + lane;
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
            int64_t lo = b0 + 31, hi = na;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (t_off[mid] <= e) lo = mid;
                else hi = mid;
            }
            b = lo;
        }
        const int64_t l = e - t_off[b];
        float s[MR], c[MR];
#pragma unroll
        for (int r = 0; r < MR; ++r) s[r] = c[r] = 0.0f;
        for (int64_t q = bcolptr[b]; q < bcolptr[b + 1]; ++q) {
            const float4 *pp = reinterpret_cast<const float4 *>(P + (pofs[q] + l) * MR);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 v = __ldg(pp + k);
                dadd(s[2 * k], c[2 * k], v.x, v.y);
                dadd(s[2 * k + 1], c[2 * k + 1], v.z, v.w);
            }
        }
        float h[MR], lo[MR];
#pragma unroll
        for (int r = 0; r < MR; ++r) norm2(s[r], c[r], h[r], lo[r]);
        float4 *th = reinterpret_cast<float4 *>(Th + e * MR), *tl = reinterpret_cast<float4 *>(Tl + e * MR);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            th[k] = make_float4(h[4 * k], h[4 * k + 1], h[4 * k + 2], h[4 * k + 3]);
            tl[k] = make_float4(lo[4 * k], lo[4 * k + 1], lo[4 * k + 2], lo[4 * k + 3]);
        }
    }
}

// ---------------------------------------------------------------------------
// row pass: Y[r0 + i][r] = sum_k D[i][k] x_r[colidx k] + sum_k U[i][k] t_r[tidx k]
// One CTA per leaf row cluster (tiles of TR rows), TR x KS threads: thread
// (i, g) accumulates row i over the columns k = g, g + KS, ... of each
// chunk of KC columns and splits the FP64 entries it uses itself (each
// entry is used by one thread).  The chunks of both panels stream through two
// shared-memory buffers by cp.async: the FP64 panel rows ([TR][AST] doubles,
// zeros past the panel) and the gathered rows of x or t ([KC][hi 16, lo
// 16]); a chunk's copies are issued while the previous one is multiplied,
// its gather indices one chunk earlier.  The KS partial sums of a row are
// added in increasing g.
// ---------------------------------------------------------------------------
constexpr int KC = 32;
constexpr int AST = KC + 2;  // doubles per staged panel row (16-byte aligned rows)

template <int TR, int KS> struct RowCfg {
    static constexpr int NT = TR * KS;
    static constexpr int ABYTES = TR * AST * 8;
    static constexpr int BUF = ABYTES + KC * 8 * 16;
    static constexpr int PA = (TR * KC / 2 + NT - 1) / NT;  // 16-byte panel pieces per thread and chunk
    static constexpr int RED = KS * TR * MR * 8;
    static constexpr int SMEM = 2 * BUF > RED ? 2 * BUF : RED;
    static_assert(NT >= KC * 8, "one gathered piece per thread and chunk");
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16(void *dst, const void *src, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr(dst)), "l"(src), "r"(pred ? 16 : 0)
                 : "memory");
}

template <int TR, int KS>
__global__ void __launch_bounds__(TR *KS, 2) row_df_kernel(
    const int32_t *__restrict__ leaf_begin, const int64_t *__restrict__ rho_off, const int32_t *__restrict__ rho_K,
    const int64_t *__restrict__ rho_colptr, const int32_t *__restrict__ colidx, const double *__restrict__ dense,
    const int64_t *__restrict__ up_off, const int32_t *__restrict__ up_K, const int64_t *__restrict__ up_colptr,
    const int32_t *__restrict__ tidx, const double *__restrict__ up, const float *__restrict__ Xh,
    const float *__restrict__ Xl, const float *__restrict__ Th, const float *__restrict__ Tl, double *__restrict__ Y,
    const int32_t *__restrict__ order) {
    using C = RowCfg<TR, KS>;
    constexpr int NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *red = reinterpret_cast<float2 *>(smem);  // [KS][TR][MR], after the last chunk
    const int t = threadIdx.x, i = t % TR, g = t / TR;
    const int64_t rho = order ? order[blockIdx.x] : blockIdx.x;
    const int32_t r0 = leaf_begin[rho], mr = leaf_begin[rho + 1] - r0;
    const int Kd = rho_K[rho], Ku = up_K[rho];
    const int nd = (Kd + KC - 1) / KC, nc = nd + (Ku + KC - 1) / KC;
    const double *Pd = dense + rho_off[rho], *Pu = up + up_off[rho];
    const int32_t *ci = colidx + rho_colptr[rho], *ti = tidx + up_colptr[rho];
    const float4 *xh4 = reinterpret_cast<const float4 *>(Xh), *xl4 = reinterpret_cast<const float4 *>(Xl);
    const float4 *th4 = reinterpret_cast<const float4 *>(Th), *tl4 = reinterpret_cast<const float4 *>(Tl);
    const int zk = t >> 3, zq = t & 7;  // this thread's gathered piece: column zk, quarter zq (hi 0-3, lo 4-7)
    for (int r0t = 0; r0t < mr; r0t += TR) {
        const int rows = min(TR, mr - r0t);
        // gather index of chunk c for this thread's piece (-1: past the panel)
        auto zindex = [&](int c) -> int {
            const bool u = c >= nd;
            const int K = u ? Ku : Kd, k = (u ? c - nd : c) * KC + zk;
            return (t < KC * 8 && k < K) ? __ldg((u ? ti : ci) + k) : -1;
        };
        auto issue = [&](int c, int zi) {
            unsigned char *buf = smem + (c & 1) * C::BUF;
            const bool u = c >= nd;
            const int K = u ? Ku : Kd, k0 = (u ? c - nd : c) * KC;
            const double *P = (u ? Pu : Pd) + (int64_t)r0t * K;
#pragma unroll
            for (int v = 0; v < C::PA; ++v) {
                const int e = t + NT * v, row = e / (KC / 2), col = 2 * (e % (KC / 2));
                if (e < TR * KC / 2) {
                    const bool ok = row < rows && k0 + col < K;
                    cp16(buf + (row * AST + col) * 8, ok ? P + (int64_t)row * K + k0 + col : P, ok);
                }
            }
            if (t < KC * 8) {
                const float4 *z = zq < 4 ? (u ? th4 : xh4) : (u ? tl4 : xl4);
                cp16(buf + C::ABYTES + t * 16, z + (int64_t)max(zi, 0) * 4 + (zq & 3), zi >= 0);
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        };
        float s[MR], c[MR];
#pragma unroll
        for (int r = 0; r < MR; ++r) s[r] = c[r] = 0.0f;
        if (nc > 0) issue(0, zindex(0));
        int zi = nc > 1 ? zindex(1) : -1;
        for (int ch = 0; ch < nc; ++ch) {
            if (ch + 1 < nc) {
                issue(ch + 1, zi);
                if (ch + 2 < nc) zi = zindex(ch + 2);
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            }
            __syncthreads();  // chunk ch has landed for every thread
            const unsigned char *buf = smem + (ch & 1) * C::BUF;
            const double *sa = reinterpret_cast<const double *>(buf) + i * AST;
            const float4 *sz = reinterpret_cast<const float4 *>(buf + C::ABYTES);
            const int K = ch < nd ? Kd : Ku, kc = min(KC, K - (ch < nd ? ch : ch - nd) * KC);
            for (int k = g; k < kc; k += KS) {
                float ah, al;
                split(sa[k], ah, al);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 xh = sz[k * 8 + q], xl = sz[k * 8 + 4 + q];
                    dfma(s[4 * q], c[4 * q], ah, al, xh.x, xl.x);
                    dfma(s[4 * q + 1], c[4 * q + 1], ah, al, xh.y, xl.y);
                    dfma(s[4 * q + 2], c[4 * q + 2], ah, al, xh.z, xl.z);
                    dfma(s[4 * q + 3], c[4 * q + 3], ah, al, xh.w, xl.w);
                }
            }
            __syncthreads();  // every thread is done with this buffer before it is refilled
        }
        // the KS partial sums of each row, in increasing g
#pragma unroll
        for (int r = 0; r < MR; ++r) red[(g * TR + i) * MR + r] = make_float2(s[r], c[r]);
        __syncthreads();
        for (int o = t; o < TR * MR; o += NT) {
            const int ii = o / MR, r = o % MR;
            if (ii >= rows) continue;
            float2 v = red[ii * MR + r];
            for (int gg = 1; gg < KS; ++gg) {
                const float2 w = red[(gg * TR + ii) * MR + r];
                dadd(v.x, v.y, w.x, w.y);
            }
            Y[(int64_t)(r0 + r0t + ii) * MR + r] = (double)v.x + (double)v.y;
        }
        __syncthreads();  // the next tile's copies reuse this memory
    }
}

// y_r[m] (Morton, [nr][n]) or y_r[perm[m]] (original order) = alpha Y[m][r] + beta y
__global__ void scatter_kernel(const double *__restrict__ Y, int64_t n, int nr, const int32_t *__restrict__ perm,
                               double alpha, double beta, double *__restrict__ y) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nr; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / n);
        const int64_t m = e - (int64_t)r * n;
        const int64_t o = (int64_t)r * n + (perm ? perm[m] : m);
        const double v = alpha * Y[m * MR + r];
        y[o] = beta == 0.0 ? v : v + beta * y[o];
    }
}

template <int TR, int KS>
static void launch_row(const hm_matrix *A, const float *Xh, const float *Xl, const float *Th, const float *Tl,
                       double *Y, const int32_t *ord, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    using C = RowCfg<TR, KS>;
    auto kern = row_df_kernel<TR, KS>;
    HM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    Trace trace("row_df_kernel", s);
    kern<<<(unsigned)tr->n_leaf, C::NT, C::SMEM, s>>>(
        tr->leaf_begin.as<int32_t>(), tr->rho_off.as<int64_t>(), tr->rho_K.as<int32_t>(), tr->rho_colptr.as<int64_t>(),
        tr->colidx.as<int32_t>(), A->dense.as<double>(), A->up_off.as<int64_t>(), A->up_K.as<int32_t>(),
        A->up_colptr.as<int64_t>(), A->tidx.as<int32_t>(), A->up.as<double>(), Xh, Xl, Th, Tl, Y, ord);
    HM_LAUNCH_CHECK();
}

// blocks of 256 threads for a grid-stride loop over n items
static unsigned grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 65535LL * 8));
}

}  // namespace df

// floats of the working arrays of one 16-right-hand-side pass: x pairs
// (2 x 16 n), partials (2 x 16 P), t pairs (2 x 16 K), Y (16 n doubles)
int64_t df_work_floats(const hm_matrix *A) {
    const int64_t n = A->tree->n, K = std::max<int64_t>(A->total_rank, 1), P = std::max<int64_t>(A->n_partials, 1);
    return 32 * n + 32 * P + 32 * K + 32 * n;
}

// Y (Morton [n][16] FP64) = H_64 x for the nr <= 16 vectors x_r = x[r * n +
// (perm ? perm[m] : m)] (Morton order without perm, original with it), in
// double-float arithmetic; work: df_work_floats(A) floats (16-byte aligned).
void matvec_df_block(const hm_matrix *A, const double *x, int nr, const int32_t *perm, double *Y, float *work,
                     cudaStream_t s) {
    using namespace df;
    const hm_tree *tr = A->tree;
    const int64_t n = tr->n, K = std::max<int64_t>(A->total_rank, 1), P = std::max<int64_t>(A->n_partials, 1);
    float *Xh = work, *Xl = Xh + MR * n;
    float2 *Pp = reinterpret_cast<float2 *>(Xl + MR * n);
    float *Th = reinterpret_cast<float *>(Pp + MR * P), *Tl = Th + MR * K;
    split_x_kernel<<<grid_for(n * MR), 256, 0, s>>>(x, n, nr, perm, Xh, Xl);
    HM_LAUNCH_CHECK();
    const int32_t *ord = A->mv_order.as<int32_t>();
    const int64_t nl = tr->n_leaf;
    if (tr->n_adm > 0) {
        {
            Trace trace("col_df_kernel", s);
            col_df_kernel<<<(unsigned)nl, CD_THREADS, 0, s>>>(
                tr->leaf_begin.as<int32_t>(), A->wp_off.as<int64_t>(), A->wp_K.as<int32_t>(),
                A->wp_colptr.as<int64_t>(), A->wp.as<double>(), Xh, Xl, Pp, ord ? ord + nl : nullptr);
            HM_LAUNCH_CHECK();
        }
        Trace trace("tsum_df_kernel", s);
        tsum_df_kernel<<<grid_for((A->total_rank + 31) / 32 * 32), 256, 0, s>>>(
            tr->n_adm, A->total_rank, A->tsum_b0.as<int32_t>(), A->t_off.as<int64_t>(), tr->lr_bcolptr.as<int64_t>(),
            A->pofs.as<int64_t>(), Pp, Th, Tl);
        HM_LAUNCH_CHECK();
    }
    if (tr->max_leaf <= 40) launch_row<40, 8>(A, Xh, Xl, Th, Tl, Y, ord, s);
    else if (tr->max_leaf <= 80) launch_row<80, 4>(A, Xh, Xl, Th, Tl, Y, ord, s);
    else launch_row<128, 2>(A, Xh, Xl, Th, Tl, Y, ord, s);
}

// y = alpha H_64 x + beta y for nrhs right-hand sides [nrhs][n] in the
// original order, 16 at a time (hm_matvec_block with HM_F64)
void matvec_df(const hm_matrix *A, int nrhs, const double *x, double *y, double alpha, double beta, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t n = tr->n;
    for (int r0 = 0; r0 < nrhs; r0 += df::MR) {
        const int nr = std::min(df::MR, nrhs - r0);
        SBuf buf;
        buf.alloc(sizeof(float) * df_work_floats(A), s);
        float *work = buf.as<float>();
        double *Y = reinterpret_cast<double *>(work + df_work_floats(A) - 32 * n);
        matvec_df_block(A, x + (int64_t)r0 * n, nr, tr->perm.as<int32_t>(), Y, work, s);
        df::scatter_kernel<<<df::grid_for(n * nr), 256, 0, s>>>(Y, n, nr, tr->perm.as<int32_t>(), alpha, beta,
                                                            y + (int64_t)r0 * n);
        HM_LAUNCH_CHECK();
    }
}

// yv (Morton [nr][n]) = H_64 xv (Morton [nr][n]) for nr <= 16 vectors
void matvec_df_morton(const hm_matrix *A, const double *xv, int nr, double *yv, float *work, cudaStream_t s) {
    const int64_t n = A->tree->n;
    double *Y = reinterpret_cast<double *>(work + df_work_floats(A) - 32 * n);
    matvec_df_block(A, xv, nr, nullptr, Y, work, s);
    df::scatter_kernel<<<df::grid_for(n * nr), 256, 0, s>>>(Y, n, nr, nullptr, 1.0, 0.0, yv);
    HM_LAUNCH_CHECK();
}

}  // namespace hm
