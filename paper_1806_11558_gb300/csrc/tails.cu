// tails.cu -- FP32 factors with BF16 tails for the 16-right-hand-side
// product of the inner solves (an option of the FP32 copy of the ACA
// factors, Sec. 2.3 and the mixed-precision iterative refinement).
//
// ACA (Sec. 2.3) builds a block as a sum of rank-one terms u_l w_l^T whose
// sizes ||u_l|| ||w_l|| fall roughly geometrically from the first term to
// the stopping tolerance.  The tensor-core product multiplies FP32 factors as
// BF16 pairs (hi + lo, about 16 significant bits: a relative error of ~2^-17
// per entry).  A term whose size is below 2^-bits of the block's largest
// term contributes at most 2^-bits of that term; rounded to BF16 (2^-9
// relative) its error is at most 2^-(9 + bits) of the largest term, below the
// pair rounding of the leading terms for bits >= 8.  So with
// factor_tail_bits = bits every block keeps its leading terms in FP32 and
// the trailing ones (from the first term after the last one at or above the
// threshold) in BF16: half the bytes for those columns of the U panels (row
// pass) and of the block-column W panels (column pass).
//
//   term_split_kernel : per block computed by the ACA, k32_b = 1 + the last
//                       term with ||u_l|| ||w_l|| >= 2^-bits max_l (FP64 sums
//                       of squares, one warp per block, fixed order);
//                       mirrored blocks take their partner's split;
//   tail_pack_kernel  : the row panels of the two parts (FP32 / BF16), from
//                       the FP64 master's row panels, in the same layout
//                       (per leaf row cluster a row-major |rho| x K panel,
//                       blocks side by side in the order of the master, widths
//                       rounded up to 8) with the t index of every column.
// The block-column W panels of the two parts are built with the other
// multi-RHS panels (mrhs.cu) from rank32 / rank16.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "hm_internal.cuh"

namespace hm {

namespace {

unsigned tgrid(int64_t n, int threads = 256) {
    const int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 65535LL * 8));
}

constexpr int TS_WARPS = 8;
constexpr int TS_MAXK = 128;  // aca_kmax <= 128

__device__ __forceinline__ bool mirrored(const int32_t *adm, const int32_t *tp, int64_t b) {
    return tp[b] >= 0 && adm[4 * b] > adm[4 * b + 2];
}

// One warp per block.  U_b: column-major m x k at uw + uw_off[b], W_b:
// row-major n x k after it.  Mirrored blocks are skipped here (their factors
// are the partner's).
__global__ void __launch_bounds__(32 * TS_WARPS)
    term_split_kernel(const int32_t *__restrict__ adm, const int32_t *__restrict__ tp,
                      const int32_t *__restrict__ rank, const int64_t *__restrict__ uw_off,
                      const double *__restrict__ uw, int64_t na, double thr2, int32_t *__restrict__ rank32) {
    __shared__ double s_u[TS_WARPS][TS_MAXK];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t b = (int64_t)blockIdx.x * TS_WARPS + w; b < na; b += (int64_t)gridDim.x * TS_WARPS) {
        if (mirrored(adm, tp, b)) continue;
        const int k = rank[b];
        if (k <= 0) {
            if (lane == 0) rank32[b] = 0;
            continue;
        }
        const int m = adm[4 * b + 1] - adm[4 * b], n = adm[4 * b + 3] - adm[4 * b + 2];
        const double *U = uw + uw_off[b];
        const double *W = U + (int64_t)m * k;
        // ||u_l||^2: lanes over the rows, one warp sum per term
        for (int l = 0; l < k; ++l) {
            double a = 0.0;
            for (int i = lane; i < m; i += 32) a = fma(U[(int64_t)l * m + i], U[(int64_t)l * m + i], a);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) s_u[w][l] = a;
        }
        __syncwarp();
        // ||w_l||^2: lanes over the terms (l = lane + 32 c), rows in order
        double sw[TS_MAXK / 32];
#pragma unroll
        for (int c = 0; c < TS_MAXK / 32; ++c) sw[c] = 0.0;
        for (int j = 0; j < n; ++j) {
#pragma unroll
            for (int c = 0; c < TS_MAXK / 32; ++c) {
                const int l = lane + 32 * c;
                if (l < k) sw[c] = fma(W[(int64_t)j * k + l], W[(int64_t)j * k + l], sw[c]);
            }
        }
        // squared sizes of this lane's terms, the largest over the block
        double mx = 0.0;
#pragma unroll
        for (int c = 0; c < TS_MAXK / 32; ++c) {
            const int l = lane + 32 * c;
            sw[c] = l < k ? s_u[w][l] * sw[c] : 0.0;
            mx = fmax(mx, sw[c]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        // the last term at or above the threshold
        int last = -1;
#pragma unroll
        for (int c = 0; c < TS_MAXK / 32; ++c) {
            const int l = lane + 32 * c;
            if (l < k && sw[c] >= thr2 * mx) last = l;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
        if (lane == 0) rank32[b] = mx > 0.0 ? last + 1 : k;
        __syncwarp();
    }
}

// per block: trailing terms, their U entries (k16 m) and all their factor
// entries (k16 (m + n)), as three int64 rows of length na + 1 (last 0) for
// the scans of the totals
__global__ void tail_count_kernel(const int32_t *__restrict__ adm, const int32_t *__restrict__ rank16, int64_t na,
                                  int64_t *__restrict__ out) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= na; b += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = 0, m = 0, n = 0;
        if (b < na) {
            k = rank16[b];
            m = adm[4 * b + 1] - adm[4 * b];
            n = adm[4 * b + 3] - adm[4 * b + 2];
        }
        out[b] = k;
        out[(na + 1) + b] = k * m;
        out[2 * (na + 1) + b] = k * (m + n);
    }
}

// mirrored blocks take their partner's split; rank16 = k - k32
__global__ void term_split_mirror_kernel(const int32_t *__restrict__ adm, const int32_t *__restrict__ tp,
                                         const int32_t *__restrict__ rank, int64_t na, int32_t *__restrict__ rank32,
                                         int32_t *__restrict__ rank16) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x) {
        if (mirrored(adm, tp, b)) rank32[b] = rank32[tp[b]];
        rank16[b] = rank[b] - rank32[b];
    }
}

// per leaf row cluster: the first column of every block in each part and the
// parts' padded widths (multiples of 8; 0 without terms) and sizes
__global__ void tail_width_kernel(const int32_t *__restrict__ leaf_begin, int64_t nleaf,
                                  const int64_t *__restrict__ lr_rowptr, const int32_t *__restrict__ lr_list,
                                  const int32_t *__restrict__ rank32, const int32_t *__restrict__ rank16,
                                  int32_t *__restrict__ koff32, int32_t *__restrict__ koff16, int32_t *__restrict__ K32,
                                  int32_t *__restrict__ K16, int64_t *__restrict__ cnt, int64_t nl1) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nleaf; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t a32 = 0, a16 = 0;
        for (int64_t q = lr_rowptr[r]; q < lr_rowptr[r + 1]; ++q) {
            const int32_t b = lr_list[q];
            koff32[q] = (int32_t)a32;
            koff16[q] = (int32_t)a16;
            a32 += rank32[b];
            a16 += rank16[b];
        }
        const int64_t p32 = (a32 + 7) / 8 * 8, p16 = (a16 + 7) / 8 * 8, mr = leaf_begin[r + 1] - leaf_begin[r];
        K32[r] = (int32_t)p32;
        K16[r] = (int32_t)p16;
        cnt[0 * nl1 + r] = mr * p32;  // entries
        cnt[1 * nl1 + r] = p32;       // columns
        cnt[2 * nl1 + r] = mr * p16;
        cnt[3 * nl1 + r] = p16;
    }
}

// The two parts of leaf row cluster r's U panel, from the master's panel
// (b's terms at columns up_koff[q] ... of it): terms l < k32_b to the FP32
// panel, the rest to the BF16 panel, zeros in the padding columns; t index
// of every column (0 for the padding, whose panel entries are zero).
__global__ void tail_pack_kernel(const int32_t *__restrict__ leaf_begin, const int64_t *__restrict__ lr_rowptr,
                                 const int32_t *__restrict__ lr_list, const int32_t *__restrict__ rank,
                                 const int32_t *__restrict__ rank32, const int64_t *__restrict__ t_off,
                                 const double *__restrict__ up, const int64_t *__restrict__ up_off,
                                 const int32_t *__restrict__ up_K, const int32_t *__restrict__ up_koff,
                                 const int32_t *__restrict__ koff32, const int32_t *__restrict__ koff16,
                                 const int32_t *__restrict__ K32, const int32_t *__restrict__ K16,
                                 const int64_t *__restrict__ off32, const int64_t *__restrict__ off16,
                                 const int64_t *__restrict__ cp32, const int64_t *__restrict__ cp16,
                                 float *__restrict__ P32, __nv_bfloat16 *__restrict__ P16, int32_t *__restrict__ ti32,
                                 int32_t *__restrict__ ti16) {
    const int64_t r = blockIdx.x;
    const int32_t mr = leaf_begin[r + 1] - leaf_begin[r];
    const int Ku = up_K[r], Ka = K32[r], Kb = K16[r];
    const double *Q = up + up_off[r];
    float *A32 = P32 + off32[r];
    __nv_bfloat16 *A16 = P16 + off16[r];
    int32_t *t32 = ti32 + cp32[r], *t16 = ti16 + cp16[r];
    const int64_t qa = lr_rowptr[r], qb = lr_rowptr[r + 1];
    for (int64_t q = qa; q < qb; ++q) {
        const int32_t b = lr_list[q];
        const int k = rank[b], k32 = rank32[b], c = up_koff[q], ca = koff32[q], cb = koff16[q];
        for (int e = threadIdx.x; e < mr * k; e += blockDim.x) {
            const int i = e / k, l = e - (e / k) * k;
            const double v = Q[(int64_t)i * Ku + c + l];
            if (l < k32) A32[(int64_t)i * Ka + ca + l] = (float)v;
            else A16[(int64_t)i * Kb + cb + (l - k32)] = __double2bfloat16(v);
        }
        for (int l = threadIdx.x; l < k; l += blockDim.x) {
            if (l < k32) t32[ca + l] = (int32_t)(t_off[b] + l);
            else t16[cb + (l - k32)] = (int32_t)(t_off[b] + l);
        }
    }
    // padding columns
    int wa = 0, wb = 0;
    if (qb > qa) {
        const int32_t b = lr_list[qb - 1];
        wa = koff32[qb - 1] + rank32[b];
        wb = koff16[qb - 1] + (rank[b] - rank32[b]);
    }
    const int pa = Ka - wa, pb = Kb - wb;
    for (int e = threadIdx.x; e < mr * pa; e += blockDim.x) {
        const int i = e / pa;
        A32[(int64_t)i * Ka + wa + (e - i * pa)] = 0.0f;
    }
    for (int e = threadIdx.x; e < mr * pb; e += blockDim.x) {
        const int i = e / pb;
        A16[(int64_t)i * Kb + wb + (e - i * pb)] = __float2bfloat16_rn(0.0f);
    }
    for (int l = threadIdx.x; l < pa; l += blockDim.x) t32[wa + l] = 0;
    for (int l = threadIdx.x; l < pb; l += blockDim.x) t16[wb + l] = 0;
}

}  // namespace

// k32 / k16 of every admissible block from the ACA's factors (uw: per block
// U_b column-major then W_b row-major at uw_off[b]; mirrored blocks share
// their partner's offset).  Sets A->rank32, A->rank16 and the info count.
void split_terms(hm_matrix *A, const DBuf &uw, const DBuf &uw_off, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t na = tr->n_adm;
    const int bits = A->params.factor_tail_bits;
    A->rank32.alloc(sizeof(int32_t) * std::max<int64_t>(na, 1));
    A->rank16.alloc(sizeof(int32_t) * std::max<int64_t>(na, 1));
    A->info.factor_tail_terms = A->info.u_tail_entries = A->info.lr_tail_entries = 0;
    if (na == 0) return;
    const double thr = std::ldexp(1.0, -bits);
    const int64_t nblk = std::min<int64_t>((na + TS_WARPS - 1) / TS_WARPS, 152LL * 64);
    term_split_kernel<<<(unsigned)nblk, 32 * TS_WARPS, 0, s>>>(tr->adm.as<int32_t>(), tr->adm_tp.as<int32_t>(),
                                                               A->rank.as<int32_t>(), uw_off.as<int64_t>(),
                                                               uw.as<double>(), na, thr * thr, A->rank32.as<int32_t>());
    HM_LAUNCH_CHECK();
    term_split_mirror_kernel<<<tgrid(na), 256, 0, s>>>(tr->adm.as<int32_t>(), tr->adm_tp.as<int32_t>(),
                                                        A->rank.as<int32_t>(), na, A->rank32.as<int32_t>(),
                                                        A->rank16.as<int32_t>());
    HM_LAUNCH_CHECK();
    DBuf c64;
    c64.alloc(sizeof(int64_t) * 3 * (na + 1));
    tail_count_kernel<<<tgrid(na + 1), 256, 0, s>>>(tr->adm.as<int32_t>(), A->rank16.as<int32_t>(), na,
                                                     c64.as<int64_t>());
    HM_LAUNCH_CHECK();
    int64_t *c = c64.as<int64_t>();
    A->info.factor_tail_terms = exclusive_scan_i64(c, c, na + 1, s);
    A->info.u_tail_entries = exclusive_scan_i64(c + (na + 1), c + (na + 1), na + 1, s);
    A->info.lr_tail_entries = exclusive_scan_i64(c + 2 * (na + 1), c + 2 * (na + 1), na + 1, s);
}

// The row panels of the two parts (with the FP32 copy; A->rank32 set).
void build_tail_panels(hm_matrix *A, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t nl = tr->n_leaf, nl1 = nl + 1;
    const int64_t nq = std::max<int64_t>(read_scalar(tr->lr_rowptr.as<int64_t>() + nl, s), 1);
    DBuf koff32, koff16, cnt, cx;
    koff32.alloc(sizeof(int32_t) * nq);
    koff16.alloc(sizeof(int32_t) * nq);
    cnt.alloc(sizeof(int64_t) * 4 * nl1);
    cx.alloc(sizeof(int64_t) * 4 * nl1);
    TailPanels &P = A->ut32, &R = A->ut16;
    P.K.alloc(sizeof(int32_t) * std::max<int64_t>(nl, 1));
    R.K.alloc(sizeof(int32_t) * std::max<int64_t>(nl, 1));
    tail_width_kernel<<<tgrid(nl), 256, 0, s>>>(tr->leaf_begin.as<int32_t>(), nl, tr->lr_rowptr.as<int64_t>(),
                                                 tr->lr_list.as<int32_t>(), A->rank32.as<int32_t>(),
                                                 A->rank16.as<int32_t>(), koff32.as<int32_t>(), koff16.as<int32_t>(),
                                                 P.K.as<int32_t>(), R.K.as<int32_t>(), cnt.as<int64_t>(), nl1);
    HM_LAUNCH_CHECK();
    HM_CUDA_CHECK(cudaMemsetAsync(cnt.as<int64_t>() + nl, 0, sizeof(int64_t), s));
    HM_CUDA_CHECK(cudaMemsetAsync(cnt.as<int64_t>() + nl1 + nl, 0, sizeof(int64_t), s));
    HM_CUDA_CHECK(cudaMemsetAsync(cnt.as<int64_t>() + 2 * nl1 + nl, 0, sizeof(int64_t), s));
    HM_CUDA_CHECK(cudaMemsetAsync(cnt.as<int64_t>() + 3 * nl1 + nl, 0, sizeof(int64_t), s));
    int64_t tot[4];
    for (int q = 0; q < 4; ++q)
        tot[q] = exclusive_scan_i64(cnt.as<int64_t>() + q * nl1, cx.as<int64_t>() + q * nl1, nl1, s);
    P.entries = tot[0];
    R.entries = tot[2];
    P.off.alloc(sizeof(int64_t) * nl1);
    P.colptr.alloc(sizeof(int64_t) * nl1);
    R.off.alloc(sizeof(int64_t) * nl1);
    R.colptr.alloc(sizeof(int64_t) * nl1);
    HM_CUDA_CHECK(cudaMemcpyAsync(P.off.p, cx.as<int64_t>(), sizeof(int64_t) * nl1, cudaMemcpyDeviceToDevice, s));
    HM_CUDA_CHECK(
        cudaMemcpyAsync(P.colptr.p, cx.as<int64_t>() + nl1, sizeof(int64_t) * nl1, cudaMemcpyDeviceToDevice, s));
    HM_CUDA_CHECK(
        cudaMemcpyAsync(R.off.p, cx.as<int64_t>() + 2 * nl1, sizeof(int64_t) * nl1, cudaMemcpyDeviceToDevice, s));
    HM_CUDA_CHECK(
        cudaMemcpyAsync(R.colptr.p, cx.as<int64_t>() + 3 * nl1, sizeof(int64_t) * nl1, cudaMemcpyDeviceToDevice, s));
    P.data.alloc(sizeof(float) * std::max<int64_t>(tot[0], 8));
    R.data.alloc(sizeof(__nv_bfloat16) * std::max<int64_t>(tot[2], 8));
    P.tidx.alloc(sizeof(int32_t) * std::max<int64_t>(tot[1], 8));
    R.tidx.alloc(sizeof(int32_t) * std::max<int64_t>(tot[3], 8));
    if (nl > 0 && tr->n_adm > 0) {
        tail_pack_kernel<<<(unsigned)nl, 256, 0, s>>>(
            tr->leaf_begin.as<int32_t>(), tr->lr_rowptr.as<int64_t>(), tr->lr_list.as<int32_t>(),
            A->rank.as<int32_t>(), A->rank32.as<int32_t>(), A->t_off.as<int64_t>(), A->up.as<double>(),
            A->up_off.as<int64_t>(), A->up_K.as<int32_t>(), A->up_koff.as<int32_t>(), koff32.as<int32_t>(),
            koff16.as<int32_t>(), P.K.as<int32_t>(), R.K.as<int32_t>(), P.off.as<int64_t>(), R.off.as<int64_t>(),
            P.colptr.as<int64_t>(), R.colptr.as<int64_t>(), P.data.as<float>(), R.data.as<__nv_bfloat16>(),
            P.tidx.as<int32_t>(), R.tidx.as<int32_t>());
        HM_LAUNCH_CHECK();
    }
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
}

}  // namespace hm
