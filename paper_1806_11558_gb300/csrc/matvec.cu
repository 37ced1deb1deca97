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
// t_b = W_b^T x_sigma, W_b row-major (n x k).  One warp per block: with
// G = floor(32 / k) lane groups, lane (g, l) accumulates column l over rows
// j = g, g + G, ..., so every load instruction reads G*k consecutive
// elements; the G partials of a column are then summed in a fixed order.
// ---------------------------------------------------------------------------
template <class TF, class TX, class TT>
__global__ void __launch_bounds__(256) lr_project_kernel(
    const int32_t *__restrict__ adm, int64_t na, const int32_t *__restrict__ rank, const int64_t *__restrict__ uw_off,
    const int64_t *__restrict__ t_off, const TF *__restrict__ uw, const TX *__restrict__ x, TT *__restrict__ t) {
    using A = typename Acc<TF>::type;
    __shared__ A s_part[8][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = w0; b < na; b += nw) {
        const int k = rank[b];
        if (k == 0) continue;
        const int32_t rb = adm[4 * b], re = adm[4 * b + 1], cb = adm[4 * b + 2], ce = adm[4 * b + 3];
        const int m = re - rb, n = ce - cb;
        const TF *W = uw + uw_off[b] + (int64_t)m * k;
        const int64_t to = t_off[b];
        for (int c0 = 0; c0 < k; c0 += 32) {
            const int kc = min(32, k - c0);
            const int G = 32 / kc;
            const int g = lane / kc, l = lane - g * kc;
            A acc = 0;
            if (g < G) {
                const TF *Wc = W + c0 + l;
                int j = g;
                for (; j + 3 * G < n; j += 4 * G) {
                    const A w0v = ld_el<TF>(Wc + (int64_t)j * k), w1v = ld_el<TF>(Wc + (int64_t)(j + G) * k);
                    const A w2v = ld_el<TF>(Wc + (int64_t)(j + 2 * G) * k), w3v = ld_el<TF>(Wc + (int64_t)(j + 3 * G) * k);
                    acc += w0v * (A)x[cb + j];
                    acc += w1v * (A)x[cb + j + G];
                    acc += w2v * (A)x[cb + j + 2 * G];
                    acc += w3v * (A)x[cb + j + 3 * G];
                }
                for (; j < n; j += G) acc += ld_el<TF>(Wc + (int64_t)j * k) * (A)x[cb + j];
            }
            s_part[wl][lane] = acc;
            __syncwarp();
            if (lane < kc) {
                A s = 0;
                for (int q = 0; q < G; ++q) s += s_part[wl][q * kc + lane];
                t[to + c0 + lane] = (TT)s;
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// y_rho = dense panel part + low-rank part, one CTA per leaf row cluster
// ---------------------------------------------------------------------------
constexpr int ROW_THREADS = 256;

template <class TD, class TF, class TX, class TT>
__global__ void __launch_bounds__(ROW_THREADS) row_kernel(
    const int32_t *__restrict__ leaf_begin, const int64_t *__restrict__ rho_off, const int32_t *__restrict__ rho_K,
    const int64_t *__restrict__ rho_colptr, const int32_t *__restrict__ colidx, const TD *__restrict__ dense,
    const int64_t *__restrict__ lr_rowptr, const LrDesc *__restrict__ desc, const TF *__restrict__ uw,
    const TT *__restrict__ t, const TX *__restrict__ x, double *__restrict__ ym) {
    using AD = typename Acc<TD>::type;
    using AF = typename Acc<TF>::type;
    __shared__ AD s_dense[MAX_LEAF];
    __shared__ AF s_lr[ROW_THREADS];
    const int64_t rho = blockIdx.x;
    const int32_t r0 = leaf_begin[rho], r1 = leaf_begin[rho + 1];
    const int mr = r1 - r0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = ROW_THREADS / 32;
    // dense near field: warp per row of rho's panel, lanes along the row
    {
        const int K = rho_K[rho];
        const TD *P = dense + rho_off[rho];
        const int32_t *ci = colidx + rho_colptr[rho];
        for (int i = warp; i < mr; i += nwarp) {
            AD acc = 0;
            const TD *row = P + (int64_t)i * K;
            int k = lane;
            for (; k + 96 < K; k += 128) {
                const int c0 = ci[k], c1 = ci[k + 32], c2 = ci[k + 64], c3 = ci[k + 96];
                const AD a0 = ld_el<TD>(row + k), a1 = ld_el<TD>(row + k + 32);
                const AD a2 = ld_el<TD>(row + k + 64), a3 = ld_el<TD>(row + k + 96);
                acc += a0 * (AD)x[c0];
                acc += a1 * (AD)x[c1];
                acc += a2 * (AD)x[c2];
                acc += a3 * (AD)x[c3];
            }
            for (; k < K; k += 32) acc += ld_el<TD>(row + k) * (AD)x[ci[k]];
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
            const LrDesc d = desc[q];
            const TF *U = uw + d.uoff + i;
            const TT *tb = t + d.toff;
            int l = 0;
            for (; l + 3 < d.k; l += 4) {
                const AF u0 = ld_el<TF>(U + (int64_t)l * d.ld), u1 = ld_el<TF>(U + (int64_t)(l + 1) * d.ld);
                const AF u2 = ld_el<TF>(U + (int64_t)(l + 2) * d.ld), u3 = ld_el<TF>(U + (int64_t)(l + 3) * d.ld);
                acc += u0 * (AF)tb[l];
                acc += u1 * (AF)tb[l + 1];
                acc += u2 * (AF)tb[l + 2];
                acc += u3 * (AF)tb[l + 3];
            }
            for (; l < d.k; ++l) acc += ld_el<TF>(U + (int64_t)l * d.ld) * (AF)tb[l];
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

// descriptors of the (leaf row cluster, admissible block) pairs
__global__ void lr_desc_kernel(const int32_t *leaf_begin, int64_t nleaf, const int64_t *lr_rowptr,
                               const int32_t *lr_list, const int32_t *adm, const int32_t *rank, const int64_t *uw_off,
                               const int64_t *t_off, LrDesc *desc) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nleaf; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r0 = leaf_begin[r];
        for (int64_t q = lr_rowptr[r]; q < lr_rowptr[r + 1]; ++q) {
            const int32_t b = lr_list[q];
            LrDesc d;
            d.uoff = uw_off[b] + (r0 - adm[4 * b]);
            d.toff = t_off[b];
            d.ld = adm[4 * b + 1] - adm[4 * b];
            d.k = rank[b];
            desc[q] = d;
        }
    }
}

__global__ void round_f32_kernel(const double *a, int64_t n, float *o) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)a[i];
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

void build_lr_desc(hm_matrix *A, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t np = read_scalar(tr->lr_rowptr.as<int64_t>() + tr->n_leaf, s);
    A->lr_desc.alloc(sizeof(LrDesc) * std::max<int64_t>(np, 1));
    if (np == 0) return;
    lr_desc_kernel<<<grid1d(tr->n_leaf), 256, 0, s>>>(tr->leaf_begin.as<int32_t>(), tr->n_leaf,
                                                     tr->lr_rowptr.as<int64_t>(), tr->lr_list.as<int32_t>(),
                                                     tr->adm.as<int32_t>(), A->rank.as<int32_t>(),
                                                     A->uw_off.as<int64_t>(), A->t_off.as<int64_t>(),
                                                     A->lr_desc.as<LrDesc>());
    HM_LAUNCH_CHECK();
}

template <class TD, class TF, class TX, class TT>
static void matvec_impl(const hm_matrix *A, const TD *dense, const TF *uw, const TX *x, TT *t, double *ym,
                        cudaStream_t s) {
    const hm_tree *tr = A->tree;
    if (tr->n_adm > 0) {
        const int64_t warps = tr->n_adm;
        lr_project_kernel<TF, TX, TT><<<grid1d(warps * 32), 256, 0, s>>>(
            tr->adm.as<int32_t>(), tr->n_adm, A->rank.as<int32_t>(), A->uw_off.as<int64_t>(),
            A->t_off.as<int64_t>(), uw, x, t);
        HM_LAUNCH_CHECK();
    }
    row_kernel<TD, TF, TX, TT><<<(unsigned)tr->n_leaf, ROW_THREADS, 0, s>>>(
        tr->leaf_begin.as<int32_t>(), tr->rho_off.as<int64_t>(), tr->rho_K.as<int32_t>(),
        tr->rho_colptr.as<int64_t>(), tr->colidx.as<int32_t>(), dense, tr->lr_rowptr.as<int64_t>(),
        A->lr_desc.as<LrDesc>(), uw, t, x, ym);
    HM_LAUNCH_CHECK();
}

// w.ym = H w.xm in Morton order.  FP64 uses w.t; the low-precision copies use
// w.x32 (x rounded once) and w.t32, with FP32 accumulation.
void matvec_morton(const hm_matrix *A, hm_dtype prec, const MatvecWork &w, cudaStream_t s) {
    const int64_t n = A->tree->n;
    switch (prec) {
        case HM_F64:
            matvec_impl<double, double, double, double>(A, A->dense.as<double>(), A->uw.as<double>(), w.xm, w.t, w.ym,
                                                        s);
            break;
        case HM_F32:
        case HM_BF16:
            if (!A->dense32.p || (prec == HM_F32 ? !A->uw32.p : !A->uwbf.p))
                fail(HM_EINVAL, "the low-precision copies for this precision were not assembled");
            round_f32_kernel<<<grid1d(n), 256, 0, s>>>(w.xm, n, w.x32);
            HM_LAUNCH_CHECK();
            if (prec == HM_F32)
                matvec_impl<float, float, float, float>(A, A->dense32.as<float>(), A->uw32.as<float>(), w.x32, w.t32,
                                                        w.ym, s);
            else
                matvec_impl<float, __nv_bfloat16, float, float>(A, A->dense32.as<float>(), A->uwbf.as<__nv_bfloat16>(),
                                                                w.x32, w.t32, w.ym, s);
            break;
        default:
            fail(HM_EINVAL, "unknown precision %d", (int)prec);
    }
}

// Device workspace of hm_matvec / the solver: xm, ym [n], t [total_rank]
// doubles, then x32 [n] and t32 [total_rank] floats.
int64_t matvec_work_doubles(const hm_matrix *A) {
    const int64_t n = A->tree->n, r = std::max<int64_t>(A->total_rank, 1);
    return 2 * n + r + (n + 1) / 2 + (r + 1) / 2;
}

MatvecWork matvec_work_at(const hm_matrix *A, double *base) {
    const int64_t n = A->tree->n, r = std::max<int64_t>(A->total_rank, 1);
    MatvecWork w;
    w.xm = base;
    w.ym = base + n;
    w.t = base + 2 * n;
    w.x32 = reinterpret_cast<float *>(base + 2 * n + r);
    w.t32 = reinterpret_cast<float *>(base + 2 * n + r + (n + 1) / 2);
    return w;
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
// Scratch layout: the product's working vectors (x and y in Morton order,
// the projections t_b = W_b^T x, and their FP32 roundings for the
// low-precision copies): 2 n + sum_b k_b doubles plus n + sum_b k_b floats.
// Every element is written before it is read in each call, so nothing needs
// clearing between calls.  The array
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
    const int64_t need = matvec_work_doubles(A);
    if (need > NOALLOC_MAX_DOUBLES)
        fail(HM_EINVAL,
             "problem too large for the allocation-free product: needs %lld scratch doubles "
             "(3 (n + sum of ranks) / 2 + n / 2), the limit is %lld",
             (long long)need, (long long)NOALLOC_MAX_DOUBLES);
    const MatvecWork w = matvec_work_at(A, noalloc_scratch());
    for (int r = 0; r < nrhs; ++r) {
        permute_to_morton(A->tree, x + (int64_t)r * n, w.xm, s);
        matvec_morton(A, prec, w, s);
        permute_from_morton(A->tree, w.ym, alpha, beta, y + (int64_t)r * n, s);
    }
}

}  // namespace hm
