// matvec.cu -- H-matrix-vector product (Sec. 2.3): dense leaves apply their
// stored block, admissible leaves apply U_b (W_b^T x_sigma).
//
// Two passes, no floating-point atomics (results are bit-identical from run to
// run):
//   lr_project_kernel : t_b = W_b^T x_sigma for every admissible leaf (one warp
//                       per leaf, lanes stream the columns of W_b).
//   row_kernel        : one CTA per leaf row cluster rho owns y_rho:
//                       y_rho = P_rho x(colidx) + sum_{b covers rho} U_b(rho, :) t_b,
//                       where P_rho is rho's row panel of the near field (warp
//                       per row, lanes stream the row) and the low-rank part is
//                       split over (row, block-phase) threads and summed in a
//                       fixed order.
// Precisions: FP64 (master), or FP32 / BF16 copies with FP32 accumulation.
#include <cuda_bf16.h>

#include <mutex>

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
// permutations between original and Morton order
// ---------------------------------------------------------------------------
__global__ void gather_perm_kernel(const double *x, const int32_t *perm, int64_t n, double *xm) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        xm[k] = x[perm[k]];
}

__global__ void scatter_perm_kernel(const double *ym, const int32_t *perm, int64_t n, double alpha, double beta,
                                    double *y) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = perm[k];
        y[i] = beta == 0.0 ? alpha * ym[k] : alpha * ym[k] + beta * y[i];
    }
}

// ---------------------------------------------------------------------------
// t_b = W_b^T x_sigma
// ---------------------------------------------------------------------------
template <class TF>
__global__ void lr_project_kernel(const int32_t *__restrict__ adm, int64_t na, const int32_t *__restrict__ rank,
                                  const int64_t *__restrict__ uw_off, const int64_t *__restrict__ t_off,
                                  const TF *__restrict__ uw, const double *__restrict__ xm, double *__restrict__ t) {
    using A = typename Acc<TF>::type;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = w0; b < na; b += nw) {
        const int32_t rb = adm[4 * b], re = adm[4 * b + 1], cb = adm[4 * b + 2], ce = adm[4 * b + 3];
        const int m = re - rb, n = ce - cb, k = rank[b];
        const TF *W = uw + uw_off[b] + (int64_t)m * k;
        for (int l = 0; l < k; ++l) {
            A acc = 0;
            for (int j = lane; j < n; j += 32) acc += ld_el<TF>(W + (int64_t)l * n + j) * (A)xm[cb + j];
            acc = warp_reduce(acc);
            if (lane == 0) t[t_off[b] + l] = (double)acc;
        }
    }
}

// ---------------------------------------------------------------------------
// y_rho = dense panel part + low-rank part, one CTA per leaf row cluster
// ---------------------------------------------------------------------------
constexpr int ROW_THREADS = 256;

template <class TD, class TF>
__global__ void __launch_bounds__(ROW_THREADS) row_kernel(
    const int32_t *__restrict__ leaf_begin, const int64_t *__restrict__ rho_off, const int32_t *__restrict__ rho_K,
    const int64_t *__restrict__ rho_colptr, const int32_t *__restrict__ colidx, const TD *__restrict__ dense,
    const int64_t *__restrict__ lr_rowptr, const int32_t *__restrict__ lr_list, const int32_t *__restrict__ adm,
    const int32_t *__restrict__ rank, const int64_t *__restrict__ uw_off, const int64_t *__restrict__ t_off,
    const TF *__restrict__ uw, const double *__restrict__ t, const double *__restrict__ xm, double *__restrict__ ym) {
    using AD = typename Acc<TD>::type;
    using AF = typename Acc<TF>::type;
    __shared__ AD s_dense[MAX_LEAF];
    __shared__ AF s_lr[ROW_THREADS];
    const int64_t rho = blockIdx.x;
    const int32_t r0 = leaf_begin[rho], r1 = leaf_begin[rho + 1];
    const int mr = r1 - r0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = ROW_THREADS / 32;
    // dense near field: warp per row
    {
        const int K = rho_K[rho];
        const TD *P = dense + rho_off[rho];
        const int32_t *ci = colidx + rho_colptr[rho];
        for (int i = warp; i < mr; i += nwarp) {
            AD acc = 0;
            const TD *row = P + (int64_t)i * K;
            for (int k = lane; k < K; k += 32) acc += ld_el<TD>(row + k) * (AD)xm[ci[k]];
            acc = warp_reduce(acc);
            if (lane == 0) s_dense[i] = acc;
        }
    }
    // low rank: thread (i, p) with p = phase over the blocks covering rho
    const int64_t l0 = lr_rowptr[rho], l1 = lr_rowptr[rho + 1];
    const int phases = ROW_THREADS / mr;  // >= 1 since mr <= MAX_LEAF <= ROW_THREADS
    const int i = threadIdx.x % mr, p = threadIdx.x / mr;
    AF acc = 0;
    if (p < phases) {
        for (int64_t q = l0 + p; q < l1; q += phases) {
            const int32_t b = lr_list[q];
            const int m = adm[4 * b + 1] - adm[4 * b], k = rank[b];
            const int off = r0 - adm[4 * b] + i;
            const TF *U = uw + uw_off[b];
            const double *tb = t + t_off[b];
            for (int l = 0; l < k; ++l) acc += ld_el<TF>(U + (int64_t)l * m + off) * (AF)tb[l];
        }
    }
    s_lr[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < mr) {
        AF s = 0;
        for (int q = 0; q < phases; ++q) s += s_lr[q * mr + threadIdx.x];
        ym[r0 + threadIdx.x] = (double)s_dense[threadIdx.x] + (double)s;
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static unsigned grid1d(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 65535LL * 8));
}

void permute_to_morton(const hm_tree *tr, const double *x, double *xm, cudaStream_t s) {
    gather_perm_kernel<<<grid1d(tr->n), 256, 0, s>>>(x, tr->perm.as<int32_t>(), tr->n, xm);
    HM_LAUNCH_CHECK();
}

void permute_from_morton(const hm_tree *tr, const double *ym, double alpha, double beta, double *y, cudaStream_t s) {
    scatter_perm_kernel<<<grid1d(tr->n), 256, 0, s>>>(ym, tr->perm.as<int32_t>(), tr->n, alpha, beta, y);
    HM_LAUNCH_CHECK();
}

template <class TD, class TF>
static void matvec_impl(const hm_matrix *A, const TD *dense, const TF *uw, const double *xm, double *ym, double *t,
                        cudaStream_t s) {
    const hm_tree *tr = A->tree;
    if (tr->n_adm > 0) {
        const int64_t warps = tr->n_adm;
        lr_project_kernel<TF><<<grid1d(warps * 32), 256, 0, s>>>(tr->adm.as<int32_t>(), tr->n_adm,
                                                                 A->rank.as<int32_t>(), A->uw_off.as<int64_t>(),
                                                                 A->t_off.as<int64_t>(), uw, xm, t);
        HM_LAUNCH_CHECK();
    }
    row_kernel<TD, TF><<<(unsigned)tr->n_leaf, ROW_THREADS, 0, s>>>(
        tr->leaf_begin.as<int32_t>(), tr->rho_off.as<int64_t>(), tr->rho_K.as<int32_t>(),
        tr->rho_colptr.as<int64_t>(), tr->colidx.as<int32_t>(), dense, tr->lr_rowptr.as<int64_t>(),
        tr->lr_list.as<int32_t>(), tr->adm.as<int32_t>(), A->rank.as<int32_t>(), A->uw_off.as<int64_t>(),
        A->t_off.as<int64_t>(), uw, t, xm, ym);
    HM_LAUNCH_CHECK();
}

// y_m = H x_m in Morton order; t: scratch of total_rank doubles
void matvec_morton(const hm_matrix *A, hm_dtype prec, const double *xm, double *ym, double *t, cudaStream_t s) {
    switch (prec) {
        case HM_F64:
            matvec_impl<double, double>(A, A->dense.as<double>(), A->uw.as<double>(), xm, ym, t, s);
            break;
        case HM_F32:
            if (!A->dense32.p || !A->uw32.p) fail(HM_EINVAL, "FP32 copies were not assembled");
            matvec_impl<float, float>(A, A->dense32.as<float>(), A->uw32.as<float>(), xm, ym, t, s);
            break;
        case HM_BF16:
            if (!A->dense32.p || !A->uwbf.p) fail(HM_EINVAL, "BF16 factors / FP32 near field were not assembled");
            matvec_impl<float, __nv_bfloat16>(A, A->dense32.as<float>(), A->uwbf.as<__nv_bfloat16>(), xm, ym, t, s);
            break;
        default:
            fail(HM_EINVAL, "unknown precision %d", (int)prec);
    }
}

// ---------------------------------------------------------------------------
// low-precision copies
// ---------------------------------------------------------------------------
__global__ void to_f32_kernel(const double *a, int64_t n, float *o) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)a[i];
}

__global__ void to_bf16_kernel(const double *a, int64_t n, __nv_bfloat16 *o) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = __float2bfloat16_rn((float)a[i]);
}

void make_low_copies(hm_matrix *A, cudaStream_t s) {
    const hm_assemble_params &p = A->params;
    const int64_t nd = A->tree->dense_entries, nf = A->lr_entries;
    if (p.dense_dtype == HM_F32 || p.factor_dtype != HM_F64) {
        A->dense32.alloc(sizeof(float) * std::max<int64_t>(nd, 1));
        to_f32_kernel<<<grid1d(nd), 256, 0, s>>>(A->dense.as<double>(), nd, A->dense32.as<float>());
        HM_LAUNCH_CHECK();
    }
    if (p.factor_dtype == HM_F32) {
        A->uw32.alloc(sizeof(float) * std::max<int64_t>(nf, 1));
        to_f32_kernel<<<grid1d(nf), 256, 0, s>>>(A->uw.as<double>(), nf, A->uw32.as<float>());
        HM_LAUNCH_CHECK();
    } else if (p.factor_dtype == HM_BF16) {
        A->uwbf.alloc(sizeof(__nv_bfloat16) * std::max<int64_t>(nf, 1));
        to_bf16_kernel<<<grid1d(nf), 256, 0, s>>>(A->uw.as<double>(), nf, A->uwbf.as<__nv_bfloat16>());
        HM_LAUNCH_CHECK();
    }
}

// ---------------------------------------------------------------------------
// load vector: f[s][perm[k]] = |T_k| sum_q w_q / (4 pi |x_q - p_s|)
// ---------------------------------------------------------------------------
__global__ void load_vector_kernel(const double *pt, int64_t npad, int64_t n, const int32_t *perm, const double *src,
                                   int nsrc, QuadParams qp, double *f) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double x[NQ], y[NQ], z[NQ];
        for (int q = 0; q < NQ; ++q) {
            x[q] = pt[(int64_t)q * npad + k];
            y[q] = pt[(int64_t)(7 + q) * npad + k];
            z[q] = pt[(int64_t)(14 + q) * npad + k];
        }
        const double area = pt[(int64_t)PT_AREA * npad + k];
        const int32_t i = perm[k];
        for (int s = 0; s < nsrc; ++s) {
            const double px = src[3 * s], py = src[3 * s + 1], pz = src[3 * s + 2];
            double acc = 0.0;
            for (int q = 0; q < NQ; ++q) {
                const double dx = x[q] - px, dy = y[q] - py, dz = z[q] - pz;
                acc += qp.w[q] / sqrt(dx * dx + dy * dy + dz * dz);
            }
            f[(int64_t)s * n + i] = area * acc * 0.079577471545947667884441881686257181;
        }
    }
}

void load_vector_impl(const hm_tree *tr, const double *src, int nsrc, double *f, cudaStream_t s) {
    const QuadParams qp = make_quad(1);
    load_vector_kernel<<<grid1d(tr->n), 256, 0, s>>>(tr->pt.as<double>(), tr->npad, tr->n, tr->perm.as<int32_t>(), src,
                                                     nsrc, qp, f);
    HM_LAUNCH_CHECK();
}


// ---------------------------------------------------------------------------
// H-matrix-vector product without any device allocation
//
// For callers that must not allocate device memory while they run: code that
// works inside a pre-sized memory budget (a pool-managed or fixed-footprint
// service), code running where an allocation would block or fail, or callers
// whose own allocator forbids stray cudaMalloc/cudaFree calls.  hm_matvec
// obtains its permuted input / output vectors and its low-rank projections
// from cudaMalloc on every call; this variant takes them from one file-scope
// device array instead, sized once when the library is loaded.
//
// Scratch layout (doubles): x in Morton order [n], y in Morton order [n],
// projections t_b = W_b^T x [sum_b k_b].  Every element is written before it
// is read in each call, so nothing needs clearing between calls.  The array
// is shared by every call on a device and keeps the last call's contents:
// calls whose work overlaps on the GPU (other streams, other host threads)
// race on it.
// ---------------------------------------------------------------------------
constexpr int64_t NOALLOC_MAX_DOUBLES = 2097152;  // 16 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_noalloc_mutex;

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in; the address is looked up once per device (with
// that device current) on the first call.
static double *noalloc_scratch() {
    int dev = 0;
    HM_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) fail(HM_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(HM_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    return static_cast<double *>(g_noalloc_ptr[dev]);
}

void matvec_noalloc(const hm_matrix *A, int32_t nrhs, hm_dtype prec, const double *x, double *y, double alpha,
                    double beta, cudaStream_t s) {
    const int64_t n = A->tree->n;
    const int64_t need = 2 * n + std::max<int64_t>(A->total_rank, 1);
    if (need > NOALLOC_MAX_DOUBLES)
        fail(HM_EINVAL,
             "problem too large for the allocation-free product: needs %lld scratch doubles "
             "(2 n + sum of ranks), the limit is %lld",
             (long long)need, (long long)NOALLOC_MAX_DOUBLES);
    double *base = noalloc_scratch();
    double *xm = base, *ym = base + n, *t = base + 2 * n;
    for (int r = 0; r < nrhs; ++r) {
        permute_to_morton(A->tree, x + (int64_t)r * n, xm, s);
        matvec_morton(A, prec, xm, ym, t, s);
        permute_from_morton(A->tree, ym, alpha, beta, y + (int64_t)r * n, s);
    }
}

}  // namespace hm
