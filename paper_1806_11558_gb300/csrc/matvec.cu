// matvec.cu -- H-matrix-vector product (Sec. 2.3): dense leaves apply their
// stored block, admissible leaves apply U_b (W_b^T x_sigma).
//
// The factors are regrouped after assembly so that every pass streams
// row-major panels with 16-byte loads (see hm_internal.cuh):
//   col_kernel  : per leaf column cluster kappa, x_kappa^T times the panel of
//                 W_b rows over the blocks whose columns cover kappa;
//   tsum_kernel : t_b = sum of those partials over the column clusters of b;
//   row_kernel  : per leaf row cluster rho, y_rho = (near-field panel) x(colidx)
//                 + (U_b rows panel) t(tidx), with the gathered vector staged
//                 in shared memory once per column chunk.
// No floating-point atomics: every sum has a fixed order, so results are
// bit-identical from run to run.  Precisions: FP64 (master), or FP32 / BF16
// copies with FP32 accumulation.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "hm_internal.cuh"
#include "mv_kernels.cuh"

namespace hm {

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
// packing of the ACA factors into low-rank row panels and the W arena
// ---------------------------------------------------------------------------
// per leaf row cluster: padded width of its low-rank panel and the first
// panel column of each of its (rho, block) pairs
__global__ void up_width_kernel(const int32_t *leaf_begin, int64_t nleaf, const int64_t *lr_rowptr,
                                const int32_t *lr_list, const int32_t *rank, int32_t *koff, int32_t *up_K,
                                int64_t *up_size, int64_t *up_kpad) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nleaf; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t acc = 0;
        for (int64_t q = lr_rowptr[r]; q < lr_rowptr[r + 1]; ++q) {
            koff[q] = (int32_t)acc;
            acc += rank[lr_list[q]];
        }
        const int64_t Kp = (acc + 7) / 8 * 8;
        up_K[r] = (int32_t)Kp;
        up_size[r] = (int64_t)(leaf_begin[r + 1] - leaf_begin[r]) * Kp;
        up_kpad[r] = Kp;
    }
}

// A block below the diagonal with a partner p uses p's factors transposed:
// U_b = W_p (row-major n_p x k) and W_b = U_p (column-major m_p x k).
__device__ __forceinline__ bool is_mirror(const int32_t *adm, const int32_t *tp, int32_t b) {
    return tp[b] >= 0 && adm[4 * b] > adm[4 * b + 2];
}

__global__ void up_pack_kernel(const int32_t *leaf_begin, const int64_t *lr_rowptr, const int32_t *lr_list,
                               const int32_t *adm, const int32_t *tp, const int32_t *rank, const int64_t *t_off,
                               const int64_t *uw_off, const double *uw, const int32_t *koff, const int64_t *up_off,
                               const int32_t *up_K, const int64_t *up_colptr, double *up, int32_t *tidx) {
    const int64_t r = blockIdx.x;
    const int32_t r0 = leaf_begin[r], mr = leaf_begin[r + 1] - r0;
    const int Ku = up_K[r];
    double *Q = up + up_off[r];
    int32_t *ti = tidx + up_colptr[r];
    for (int64_t q = lr_rowptr[r]; q < lr_rowptr[r + 1]; ++q) {
        const int32_t b = lr_list[q];
        const int k = rank[b], off = r0 - adm[4 * b], c = koff[q];
        if (is_mirror(adm, tp, b)) {
            const int32_t p = tp[b];
            const int mp = adm[4 * p + 1] - adm[4 * p];
            const double *Wp = uw + uw_off[p] + (int64_t)mp * k;
            for (int e = threadIdx.x; e < mr * k; e += blockDim.x) {
                const int i = e / k, l = e - (e / k) * k;
                Q[(int64_t)i * Ku + c + l] = Wp[(int64_t)(off + i) * k + l];
            }
        } else {
            const int m = adm[4 * b + 1] - adm[4 * b];
            const double *U = uw + uw_off[b];
            for (int e = threadIdx.x; e < mr * k; e += blockDim.x) {
                const int i = e / k, l = e - (e / k) * k;
                Q[(int64_t)i * Ku + c + l] = U[(int64_t)l * m + off + i];
            }
        }
        for (int l = threadIdx.x; l < k; l += blockDim.x) ti[c + l] = (int32_t)(t_off[b] + l);
    }
    // the padding columns (the panel width rounded up to 8) are zeros
    const int64_t qa = lr_rowptr[r], qb = lr_rowptr[r + 1];
    const int kw = qb > qa ? koff[qb - 1] + rank[lr_list[qb - 1]] : 0, pw = Ku - kw;
    for (int e = threadIdx.x; e < mr * pw; e += blockDim.x) {
        const int i = e / pw;
        Q[(int64_t)i * Ku + kw + (e - i * pw)] = 0.0;
    }
}

// column panels of W: per leaf column cluster kappa, W_b(rows of kappa, :)
// over the admissible leaves whose columns cover kappa
__global__ void wp_pack_kernel(const int32_t *leaf_begin, const int64_t *lr_colptr, const int32_t *lr_collist,
                               const int32_t *adm, const int32_t *tp, const int32_t *rank, const int64_t *uw_off,
                               const double *uw, const int32_t *koff, const int64_t *wp_off, const int32_t *wp_K,
                               double *wp) {
    const int64_t kap = blockIdx.x;
    const int32_t c0 = leaf_begin[kap], mc = leaf_begin[kap + 1] - c0;
    const int Kw = wp_K[kap];
    double *Wt = wp + wp_off[kap];
    for (int64_t q = lr_colptr[kap]; q < lr_colptr[kap + 1]; ++q) {
        const int32_t b = lr_collist[q];
        const int k = rank[b], off = c0 - adm[4 * b + 2], c = koff[q];
        if (is_mirror(adm, tp, b)) {
            const int32_t p = tp[b];
            const int mp = adm[4 * p + 1] - adm[4 * p];
            const double *Up = uw + uw_off[p];  // column-major m_p x k
            for (int e = threadIdx.x; e < mc * k; e += blockDim.x) {
                const int j = e / k, l = e - (e / k) * k;
                Wt[(int64_t)j * Kw + c + l] = Up[(int64_t)l * mp + off + j];
            }
        } else {
            const int m = adm[4 * b + 1] - adm[4 * b];
            const double *W = uw + uw_off[b] + (int64_t)m * k;  // row-major n x k
            for (int e = threadIdx.x; e < mc * k; e += blockDim.x) {
                const int j = e / k, l = e - (e / k) * k;
                Wt[(int64_t)j * Kw + c + l] = W[(int64_t)(off + j) * k + l];
            }
        }
    }
    // the padding columns (the panel width rounded up to 8) are zeros
    const int64_t qa = lr_colptr[kap], qb = lr_colptr[kap + 1];
    const int kw = qb > qa ? koff[qb - 1] + rank[lr_collist[qb - 1]] : 0, pw = Kw - kw;
    for (int e = threadIdx.x; e < mc * pw; e += blockDim.x) {
        const int j = e / pw;
        Wt[(int64_t)j * Kw + kw + (e - j * pw)] = 0.0;
    }
}

// offset of the partial projection of each (block, leaf cluster) pair: the
// column leaf clusters of the block (side = 2, projections through the W
// panels, product with H) or its row leaf clusters (side = 0, through the U
// panels, product with H^T)
__global__ void pofs_kernel(const int32_t *leaf_begin, int64_t nleaf, const int64_t *lr_colptr,
                            const int32_t *lr_collist, const int32_t *adm, int side, const int64_t *wp_colptr,
                            const int32_t *koff, const int64_t *bcolptr, int64_t *pofs) {
    for (int64_t kap = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; kap < nleaf;
         kap += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t q = lr_colptr[kap]; q < lr_colptr[kap + 1]; ++q) {
            const int32_t b = lr_collist[q];
            int64_t lo = 0, hi = nleaf;
            const int32_t cb = adm[4 * b + side];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (leaf_begin[mid] < cb) lo = mid + 1;
                else hi = mid;
            }
            pofs[bcolptr[b] + (kap - lo)] = wp_colptr[kap] + koff[q];
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

// Regroups the ACA output (uw: U_b column-major then W_b row-major at
// uw_off[b]) into the low-rank row panels (U) and column panels (W).
void build_lr_panels(hm_matrix *A, const DBuf &uw, const DBuf &uw_off, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t nl = tr->n_leaf, na = tr->n_adm;
    const int64_t np = read_scalar(tr->lr_rowptr.as<int64_t>() + nl, s);
    A->up_koff.alloc(sizeof(int32_t) * std::max<int64_t>(np, 1));
    A->up_K.alloc(sizeof(int32_t) * nl);
    A->up_off.alloc(sizeof(int64_t) * (nl + 1));
    A->up_colptr.alloc(sizeof(int64_t) * (nl + 1));
    DBuf size, kpad;
    size.alloc(sizeof(int64_t) * (nl + 1));
    kpad.alloc(sizeof(int64_t) * (nl + 1));
    up_width_kernel<<<grid1d(nl), 256, 0, s>>>(tr->leaf_begin.as<int32_t>(), nl, tr->lr_rowptr.as<int64_t>(),
                                              tr->lr_list.as<int32_t>(), A->rank.as<int32_t>(),
                                              A->up_koff.as<int32_t>(), A->up_K.as<int32_t>(), size.as<int64_t>(),
                                              kpad.as<int64_t>());
    HM_LAUNCH_CHECK();
    HM_CUDA_CHECK(cudaMemsetAsync(size.as<int64_t>() + nl, 0, sizeof(int64_t), s));
    HM_CUDA_CHECK(cudaMemsetAsync(kpad.as<int64_t>() + nl, 0, sizeof(int64_t), s));
    A->up_entries = exclusive_scan_i64(size.as<int64_t>(), A->up_off.as<int64_t>(), nl + 1, s);
    const int64_t ncol = exclusive_scan_i64(kpad.as<int64_t>(), A->up_colptr.as<int64_t>(), nl + 1, s);
    A->n_partials_t = ncol;  // projections through the U panels (transposed product)
    A->up.alloc(sizeof(double) * std::max<int64_t>(A->up_entries, 8));
    A->tidx.alloc(sizeof(int32_t) * std::max<int64_t>(ncol, 8));
    HM_CUDA_CHECK(cudaMemsetAsync(A->tidx.p, 0, sizeof(int32_t) * std::max<int64_t>(ncol, 8), s));
    if (na > 0 && nl > 0) {
        up_pack_kernel<<<(unsigned)nl, 256, 0, s>>>(
            tr->leaf_begin.as<int32_t>(), tr->lr_rowptr.as<int64_t>(), tr->lr_list.as<int32_t>(),
            tr->adm.as<int32_t>(), tr->adm_tp.as<int32_t>(), A->rank.as<int32_t>(), A->t_off.as<int64_t>(),
            uw_off.as<int64_t>(),
            uw.as<double>(), A->up_koff.as<int32_t>(), A->up_off.as<int64_t>(), A->up_K.as<int32_t>(),
            A->up_colptr.as<int64_t>(), A->up.as<double>(), A->tidx.as<int32_t>());
        HM_LAUNCH_CHECK();
    }
    // W column panels and the partial-projection map
    A->wp_koff.alloc(sizeof(int32_t) * std::max<int64_t>(read_scalar(tr->lr_colptr.as<int64_t>() + nl, s), 1));
    A->wp_K.alloc(sizeof(int32_t) * nl);
    A->wp_off.alloc(sizeof(int64_t) * (nl + 1));
    A->wp_colptr.alloc(sizeof(int64_t) * (nl + 1));
    up_width_kernel<<<grid1d(nl), 256, 0, s>>>(tr->leaf_begin.as<int32_t>(), nl, tr->lr_colptr.as<int64_t>(),
                                              tr->lr_collist.as<int32_t>(), A->rank.as<int32_t>(),
                                              A->wp_koff.as<int32_t>(), A->wp_K.as<int32_t>(), size.as<int64_t>(),
                                              kpad.as<int64_t>());
    HM_LAUNCH_CHECK();
    HM_CUDA_CHECK(cudaMemsetAsync(size.as<int64_t>() + nl, 0, sizeof(int64_t), s));
    HM_CUDA_CHECK(cudaMemsetAsync(kpad.as<int64_t>() + nl, 0, sizeof(int64_t), s));
    A->wp_entries = exclusive_scan_i64(size.as<int64_t>(), A->wp_off.as<int64_t>(), nl + 1, s);
    A->n_partials = exclusive_scan_i64(kpad.as<int64_t>(), A->wp_colptr.as<int64_t>(), nl + 1, s);
    A->wp.alloc(sizeof(double) * std::max<int64_t>(A->wp_entries, 8));
    const int64_t npairs = read_scalar(tr->lr_bcolptr.as<int64_t>() + na, s);
    A->pofs.alloc(sizeof(int64_t) * std::max<int64_t>(npairs, 1));
    if (na > 0 && nl > 0) {
        wp_pack_kernel<<<(unsigned)nl, 256, 0, s>>>(tr->leaf_begin.as<int32_t>(), tr->lr_colptr.as<int64_t>(),
                                                   tr->lr_collist.as<int32_t>(), tr->adm.as<int32_t>(),
                                                   tr->adm_tp.as<int32_t>(), A->rank.as<int32_t>(),
                                                   uw_off.as<int64_t>(), uw.as<double>(),
                                                   A->wp_koff.as<int32_t>(), A->wp_off.as<int64_t>(),
                                                   A->wp_K.as<int32_t>(), A->wp.as<double>());
        HM_LAUNCH_CHECK();
        pofs_kernel<<<grid1d(nl), 256, 0, s>>>(tr->leaf_begin.as<int32_t>(), nl, tr->lr_colptr.as<int64_t>(),
                                              tr->lr_collist.as<int32_t>(), tr->adm.as<int32_t>(), 2,
                                              A->wp_colptr.as<int64_t>(), A->wp_koff.as<int32_t>(),
                                              tr->lr_bcolptr.as<int64_t>(), A->pofs.as<int64_t>());
        HM_LAUNCH_CHECK();
        A->tsum_b0.alloc(sizeof(int32_t) * std::max<int64_t>((A->total_rank + 31) / 32, 1));
        if (A->total_rank > 0) {
            tsum_b0_kernel<<<grid1d(na), 256, 0, s>>>(na, A->t_off.as<int64_t>(), A->tsum_b0.as<int32_t>());
            HM_LAUNCH_CHECK();
        }
    }
    // dispatch orders of the product's kernels: leaf clusters by decreasing
    // work (rows x panel width; ties by index), forward and transposed
    if (nl > 0) {
        std::vector<int32_t> lb(nl + 1), kd(nl), ku(nl), kw(nl);
        HM_CUDA_CHECK(cudaMemcpyAsync(lb.data(), tr->leaf_begin.p, sizeof(int32_t) * (nl + 1), cudaMemcpyDeviceToHost, s));
        HM_CUDA_CHECK(cudaMemcpyAsync(kd.data(), tr->rho_K.p, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, s));
        HM_CUDA_CHECK(cudaMemcpyAsync(ku.data(), A->up_K.p, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, s));
        HM_CUDA_CHECK(cudaMemcpyAsync(kw.data(), A->wp_K.p, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, s));
        HM_CUDA_CHECK(cudaStreamSynchronize(s));
        std::vector<int32_t> ord(4 * nl);
        auto by_work = [&](int32_t *o, auto work) {
            for (int64_t r = 0; r < nl; ++r) o[r] = (int32_t)r;
            std::stable_sort(o, o + nl, [&](int32_t a, int32_t b) { return work(a) > work(b); });
        };
        auto rows = [&](int32_t r) { return (int64_t)(lb[r + 1] - lb[r]); };
        by_work(ord.data(), [&](int32_t r) { return rows(r) * ((int64_t)kd[r] + ku[r]); });
        by_work(ord.data() + nl, [&](int32_t r) { return rows(r) * (int64_t)kw[r]; });
        by_work(ord.data() + 2 * nl, [&](int32_t r) { return rows(r) * ((int64_t)kd[r] + kw[r]); });
        by_work(ord.data() + 3 * nl, [&](int32_t r) { return rows(r) * (int64_t)ku[r]; });
        A->mv_order.alloc(sizeof(int32_t) * 4 * nl);
        HM_CUDA_CHECK(cudaMemcpyAsync(A->mv_order.p, ord.data(), sizeof(int32_t) * 4 * nl, cudaMemcpyHostToDevice, s));
        HM_CUDA_CHECK(cudaStreamSynchronize(s));
    }
}

// ---------------------------------------------------------------------------
// transposed product H^T (data built on first use)
// ---------------------------------------------------------------------------
// Near field of H^T in the layout of the row panels: the place of dense leaf
// b (rows rho_b, columns sigma_b) receives A(sigma_b, rho_b)^T.  The entries
// come from b's transposed partner when the block tree has one (always for
// Algorithm 1 on I x I with a symmetric admissibility); otherwise every
// column j of b looks up the dense leaf that holds A(cb + j, rho_b): dense
// leaves are sorted by (row begin, column begin) and their row ranges are
// leaf clusters.
constexpr int DT_MAX_COLS = 2 * MAX_LEAF;
__global__ void to_f32_kernel(const double *a, int64_t n, float *o);

__global__ void dense_transpose_kernel(const int32_t *__restrict__ dense, int64_t nd, const int64_t *__restrict__ base,
                                       const int32_t *__restrict__ ld, const int32_t *__restrict__ tp,
                                       const int32_t *__restrict__ leaf_begin, int64_t nleaf,
                                       const double *__restrict__ A, double *__restrict__ AT, int *err) {
    __shared__ int64_t s_src[DT_MAX_COLS];
    const int64_t b = blockIdx.x;
    const int32_t rb = dense[4 * b], re = dense[4 * b + 1], cb = dense[4 * b + 2], ce = dense[4 * b + 3];
    const int m = re - rb, n = ce - cb;
    const int64_t bb = base[b];
    const int32_t lb = ld[b];
    const int32_t p = tp[b];
    if (p >= 0) {
        const int64_t bp = base[p];
        const int32_t lp = ld[p];
        for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
            const int i = e / n, j = e - (e / n) * n;
            AT[bb + (int64_t)i * lb + j] = A[bp + (int64_t)j * lp + i];
        }
        return;
    }
    if (n > DT_MAX_COLS) {
        if (threadIdx.x == 0) atomicExch(err, 4);
        return;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int32_t r = cb + j;
        // leaf cluster of row r
        int64_t lo = 0, hi = nleaf;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (leaf_begin[mid] <= r) lo = mid;
            else hi = mid;
        }
        const int32_t R = leaf_begin[lo];
        // last dense leaf with (row begin, column begin) <= (R, rb)
        int64_t a = -1, z = nd;
        while (z - a > 1) {
            const int64_t mid = (a + z) >> 1;
            const int32_t mr = dense[4 * mid], mc = dense[4 * mid + 2];
            if (mr < R || (mr == R && mc <= rb)) a = mid;
            else z = mid;
        }
        int64_t src = -1;
        if (a >= 0 && dense[4 * a] == R && dense[4 * a + 1] > r && dense[4 * a + 2] <= rb && dense[4 * a + 3] >= re)
            src = base[a] + (int64_t)(r - R) * ld[a] + (rb - dense[4 * a + 2]);
        if (src < 0) atomicExch(err, 4);
        s_src[j] = src;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
        const int i = e / n, j = e - (e / n) * n;
        const int64_t src = s_src[j];
        AT[bb + (int64_t)i * lb + j] = src >= 0 ? A[src + i] : 0.0;
    }
}

// t index of every column of the W panels (padding columns keep 0)
__global__ void tidx_cols_kernel(const int64_t *lr_colptr, const int32_t *lr_collist, const int32_t *rank,
                                 const int64_t *t_off, const int32_t *wp_koff, const int64_t *wp_colptr,
                                 int32_t *tidx_t) {
    const int64_t kap = blockIdx.x;
    for (int64_t q = lr_colptr[kap]; q < lr_colptr[kap + 1]; ++q) {
        const int32_t b = lr_collist[q];
        const int k = rank[b];
        for (int l = threadIdx.x; l < k; l += blockDim.x)
            tidx_t[wp_colptr[kap] + wp_koff[q] + l] = (int32_t)(t_off[b] + l);
    }
}

void build_transposed(const hm_matrix *Ac, cudaStream_t s) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    hm_matrix *A = const_cast<hm_matrix *>(Ac);  // cache owned by the matrix
    if (A->trans_ready) return;
    const hm_tree *tr = A->tree;
    const int64_t nl = tr->n_leaf, na = tr->n_adm, nd = tr->n_dense;
    const int64_t ne = std::max<int64_t>(tr->dense_entries, 1);
    A->dense_t.alloc(sizeof(double) * ne);
    HM_CUDA_CHECK(cudaMemsetAsync(A->dense_t.p, 0, sizeof(double) * ne, s));
    DBuf err;
    err.alloc(sizeof(int));
    HM_CUDA_CHECK(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    if (nd > 0) {
        dense_transpose_kernel<<<(unsigned)nd, 128, 0, s>>>(tr->dense.as<int32_t>(), nd, tr->dense_base.as<int64_t>(),
                                                           tr->dense_ld.as<int32_t>(), tr->dense_tp.as<int32_t>(),
                                                           tr->leaf_begin.as<int32_t>(), nl, A->dense.as<double>(),
                                                           A->dense_t.as<double>(), err.as<int>());
        HM_LAUNCH_CHECK();
    }
    if (A->dense32.p) {
        A->dense32_t.alloc(sizeof(float) * ne);
        to_f32_kernel<<<grid1d(ne), 256, 0, s>>>(A->dense_t.as<double>(), ne, A->dense32_t.as<float>());
        HM_LAUNCH_CHECK();
    }
    const int64_t npairs = read_scalar(tr->lr_browptr.as<int64_t>() + na, s);
    A->pofs_t.alloc(sizeof(int64_t) * std::max<int64_t>(npairs, 1));
    A->tidx_t.alloc(sizeof(int32_t) * std::max<int64_t>(A->n_partials, 8));
    HM_CUDA_CHECK(cudaMemsetAsync(A->tidx_t.p, 0, sizeof(int32_t) * std::max<int64_t>(A->n_partials, 8), s));
    if (na > 0 && nl > 0) {
        pofs_kernel<<<grid1d(nl), 256, 0, s>>>(tr->leaf_begin.as<int32_t>(), nl, tr->lr_rowptr.as<int64_t>(),
                                              tr->lr_list.as<int32_t>(), tr->adm.as<int32_t>(), 0,
                                              A->up_colptr.as<int64_t>(), A->up_koff.as<int32_t>(),
                                              tr->lr_browptr.as<int64_t>(), A->pofs_t.as<int64_t>());
        HM_LAUNCH_CHECK();
        tidx_cols_kernel<<<(unsigned)nl, 128, 0, s>>>(tr->lr_colptr.as<int64_t>(), tr->lr_collist.as<int32_t>(),
                                                      A->rank.as<int32_t>(), A->t_off.as<int64_t>(),
                                                      A->wp_koff.as<int32_t>(), A->wp_colptr.as<int64_t>(),
                                                      A->tidx_t.as<int32_t>());
        HM_LAUNCH_CHECK();
    }
    if (read_scalar(err.as<int>(), s) != 0)
        fail(HM_EINTERNAL, "transposed near field: an entry of H^T has no stored counterpart");
    A->trans_ready = true;
}

// Trace names of the three kernels of one product, per precision
struct MvNames {
    const char *col, *tsum, *row;
};
constexpr MvNames MV_F64{"col_kernel.f64", "tsum_kernel.f64", "row_kernel.f64"};
constexpr MvNames MV_F32{"col_kernel.f32", "tsum_kernel.f32", "row_kernel.f32"};
constexpr MvNames MV_BF16{"col_kernel.bf16", "tsum_kernel.bf16", "row_kernel.bf16"};
constexpr MvNames MV_F64_T{"col_kernel.f64.t", "tsum_kernel.f64.t", "row_kernel.f64.t"};
constexpr MvNames MV_F32_T{"col_kernel.f32.t", "tsum_kernel.f32.t", "row_kernel.f32.t"};
constexpr MvNames MV_BF16_T{"col_kernel.bf16.t", "tsum_kernel.bf16.t", "row_kernel.bf16.t"};

// Index data of one direction of the product: the projection panels (one
// per leaf cluster, x_kappa^T times the panel gives the partials), the
// partial offsets of each block, and the expansion panels with the t index
// of each of their columns.  H: project through the W column panels, expand
// through the U row panels.  H^T: project through the U panels, expand
// through the W panels (U and W swap roles), near field transposed.
struct MvDir {
    const int64_t *proj_off, *proj_ptr;
    const int32_t *proj_K;
    const int64_t *bptr, *pofs;
    const int64_t *exp_off, *exp_ptr;
    const int32_t *exp_K, *exp_tidx;
    const int32_t *row_order, *col_order;
};

static MvDir mv_dir(const hm_matrix *A, bool trans) {
    const hm_tree *tr = A->tree;
    const int32_t *ord = A->mv_order.as<int32_t>();
    const int64_t nl = tr->n_leaf;
    if (!trans)
        return MvDir{A->wp_off.as<int64_t>(), A->wp_colptr.as<int64_t>(), A->wp_K.as<int32_t>(),
                     tr->lr_bcolptr.as<int64_t>(), A->pofs.as<int64_t>(), A->up_off.as<int64_t>(),
                     A->up_colptr.as<int64_t>(), A->up_K.as<int32_t>(), A->tidx.as<int32_t>(),
                     ord ? ord : nullptr, ord ? ord + nl : nullptr};
    return MvDir{A->up_off.as<int64_t>(), A->up_colptr.as<int64_t>(), A->up_K.as<int32_t>(),
                 tr->lr_browptr.as<int64_t>(), A->pofs_t.as<int64_t>(), A->wp_off.as<int64_t>(),
                 A->wp_colptr.as<int64_t>(), A->wp_K.as<int32_t>(), A->tidx_t.as<int32_t>(),
                 ord ? ord + 2 * nl : nullptr, ord ? ord + 3 * nl : nullptr};
}

template <class TD, class TF, class TX, class TT>
static void matvec_impl(const hm_matrix *A, const TD *dense, const TF *proj, const TF *expd, const MvDir &d,
                        const TX *x, TT *p, TT *t, double *ym, const MvNames &nm, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    if (tr->n_adm > 0) {
        Trace tr_col(nm.col, s);
        col_kernel<TF, TX, TT><<<(unsigned)tr->n_leaf, COL_THREADS, 0, s>>>(tr->leaf_begin.as<int32_t>(), d.proj_off,
                                                                            d.proj_K, d.proj_ptr, proj, x, p,
                                                                            d.col_order);
        HM_LAUNCH_CHECK();
    }
    if (tr->n_adm > 0) {
        Trace tr_tsum(nm.tsum, s);
        tsum_kernel<TT, TT><<<grid1d((A->total_rank + 31) / 32 * 32), 256, 0, s>>>(
            tr->n_adm, A->total_rank, A->tsum_b0.as<int32_t>(), A->t_off.as<int64_t>(), d.bptr, d.pofs, p, t);
        HM_LAUNCH_CHECK();
    }
    // the FP64 row kernel (FP64-pipe-bound) runs its clusters largest first;
    // the FP32 / BF16 one (HBM-bound) keeps the Morton order, whose
    // neighbouring clusters share their gathered x and t in L2 (measured:
    // largest-first 3.50 -> 3.28 ms in FP64, 1.24 -> 1.33 ms in FP32)
    constexpr bool ORD = sizeof(TD) == 8;
    auto kern = row_kernel<12, TD, TF, TX, TT, ORD>;
    switch (row_rb_for(tr->max_leaf)) {
        case 4: kern = row_kernel<4, TD, TF, TX, TT, ORD>; break;
        case 5: kern = row_kernel<5, TD, TF, TX, TT, ORD>; break;
        case 8: kern = row_kernel<8, TD, TF, TX, TT, ORD>; break;
        default: break;
    }
    Trace tr_row(nm.row, s);
    kern<<<(unsigned)tr->n_leaf, ROW_THREADS, 0, s>>>(
        tr->leaf_begin.as<int32_t>(), tr->rho_off.as<int64_t>(), tr->rho_K.as<int32_t>(),
        tr->rho_colptr.as<int64_t>(), tr->colidx.as<int32_t>(), dense, d.exp_off, d.exp_K, d.exp_ptr, d.exp_tidx,
        expd, t, x, ym, d.row_order);
    HM_LAUNCH_CHECK();
}

// w.ym = op(H) w.xm in Morton order.  FP64 uses w.t; the low-precision
// copies use w.x32 (x rounded once) and w.t32, with FP32 accumulation.  The
// transposed product needs build_transposed() first.
void matvec_morton(const hm_matrix *A, hm_dtype prec, const MatvecWork &w, cudaStream_t s, bool trans) {
    const int64_t n = A->tree->n;
    if (trans && !A->trans_ready) fail(HM_EINTERNAL, "transposed data not built");
    const MvDir d = mv_dir(A, trans);
    switch (prec) {
        case HM_F64: {
            const double *dn = trans ? A->dense_t.as<double>() : A->dense.as<double>();
            const double *pr = trans ? A->up.as<double>() : A->wp.as<double>();
            const double *ex = trans ? A->wp.as<double>() : A->up.as<double>();
            matvec_impl<double, double, double, double>(A, dn, pr, ex, d, w.xm, w.p, w.t, w.ym,
                                                        trans ? MV_F64_T : MV_F64, s);
            break;
        }
        case HM_F32:
        case HM_BF16: {
            if (!A->dense32.p || (prec == HM_F32 ? !A->up32.p : !A->upbf.p))
                fail(HM_EINVAL, "the low-precision copies for this precision were not assembled");
            round_f32_kernel<<<grid1d(n), 256, 0, s>>>(w.xm, n, w.x32);
            HM_LAUNCH_CHECK();
            const float *dn = trans ? A->dense32_t.as<float>() : A->dense32.as<float>();
            if (prec == HM_F32) {
                const float *pr = trans ? A->up32.as<float>() : A->wp32.as<float>();
                const float *ex = trans ? A->wp32.as<float>() : A->up32.as<float>();
                matvec_impl<float, float, float, float>(A, dn, pr, ex, d, w.x32, w.p32, w.t32, w.ym,
                                                        trans ? MV_F32_T : MV_F32, s);
            } else {
                const __nv_bfloat16 *pr = trans ? A->upbf.as<__nv_bfloat16>() : A->wpbf.as<__nv_bfloat16>();
                const __nv_bfloat16 *ex = trans ? A->wpbf.as<__nv_bfloat16>() : A->upbf.as<__nv_bfloat16>();
                matvec_impl<float, __nv_bfloat16, float, float>(A, dn, pr, ex, d, w.x32, w.p32, w.t32, w.ym,
                                                                trans ? MV_BF16_T : MV_BF16, s);
            }
            break;
        }
        default:
            fail(HM_EINVAL, "unknown precision %d", (int)prec);
    }
}

// Device workspace of hm_matvec / the solver: xm, ym [n], t [K], p [P]
// doubles, then x32 [n], t32 [K], p32 [P] floats (K = sum of ranks, P = the
// partial projections of the column panels).
// Working vectors of a product whose partial-projection vector has q entries
// (q = P for the forward product, max(P, P_T) to serve both directions).
static int64_t work_doubles(const hm_matrix *A, int64_t q) {
    const int64_t n = A->tree->n, r = std::max<int64_t>(A->total_rank, 1);
    q = std::max<int64_t>(q, 1);
    return 2 * n + r + q + (n + 1) / 2 + (r + 1) / 2 + (q + 1) / 2;
}

static MatvecWork work_at(const hm_matrix *A, double *base, int64_t q);

int64_t matvec_work_doubles(const hm_matrix *A) {
    return work_doubles(A, std::max(A->n_partials, A->n_partials_t));
}

MatvecWork matvec_work_at(const hm_matrix *A, double *base) {
    return work_at(A, base, std::max(A->n_partials, A->n_partials_t));
}

static MatvecWork work_at(const hm_matrix *A, double *base, int64_t q) {
    const int64_t n = A->tree->n, r = std::max<int64_t>(A->total_rank, 1);
    q = std::max<int64_t>(q, 1);
    MatvecWork w;
    w.xm = base;
    w.ym = base + n;
    w.t = base + 2 * n;
    w.p = base + 2 * n + r;
    double *f = base + 2 * n + r + q;
    w.x32 = reinterpret_cast<float *>(f);
    w.t32 = reinterpret_cast<float *>(f + (n + 1) / 2);
    w.p32 = reinterpret_cast<float *>(f + (n + 1) / 2 + (r + 1) / 2);
    return w;
}

// ---------------------------------------------------------------------------
// one leaf as a dense array (introspection)
// ---------------------------------------------------------------------------
__global__ void get_dense_block_kernel(const int64_t base, const int32_t ld, int m, int n, const double *dense,
                                       double *out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e - (e / n) * n);
        out[e] = dense[base + (int64_t)i * ld + j];
    }
}

__device__ __forceinline__ int64_t find_in(const int32_t *list, int64_t lo, int64_t hi, int32_t v) {
    for (; lo < hi; ++lo)  // lists are short (the blocks of one leaf cluster)
        if (list[lo] == v) break;
    return lo;
}

__device__ __forceinline__ int64_t leaf_of(const int32_t *leaf_begin, int64_t nl, int32_t row) {
    int64_t lo = 0, hi = nl;  // last leaf with begin <= row
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (leaf_begin[mid] <= row) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void get_lr_block_kernel(int32_t b, int32_t rb, int32_t cb, int m, int n, int k,
                                    const int32_t *leaf_begin, int64_t nl, const int64_t *lr_rowptr,
                                    const int32_t *lr_list, const int32_t *up_koff, const int64_t *up_off,
                                    const int32_t *up_K, const double *up, const int64_t *lr_colptr,
                                    const int32_t *lr_collist, const int32_t *wp_koff, const int64_t *wp_off,
                                    const int32_t *wp_K, const double *wp, double *out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e - (e / n) * n);
        const int64_t r = leaf_of(leaf_begin, nl, rb + i), c = leaf_of(leaf_begin, nl, cb + j);
        const int64_t qr = find_in(lr_list, lr_rowptr[r], lr_rowptr[r + 1], b);
        const int64_t qc = find_in(lr_collist, lr_colptr[c], lr_colptr[c + 1], b);
        const double *Ur = up + up_off[r] + (int64_t)(rb + i - leaf_begin[r]) * up_K[r] + up_koff[qr];
        const double *Wr = wp + wp_off[c] + (int64_t)(cb + j - leaf_begin[c]) * wp_K[c] + wp_koff[qc];
        double acc = 0.0;
        for (int l = 0; l < k; ++l) acc += Ur[l] * Wr[l];
        out[e] = acc;
    }
}

void get_block(const hm_matrix *A, int dense, int64_t b, double *out, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    const int64_t nb = dense ? tr->n_dense : tr->n_adm;
    if (b < 0 || b >= nb) fail(HM_EINVAL, "leaf index %lld out of range", (long long)b);
    int32_t q[4];
    HM_CUDA_CHECK(cudaMemcpyAsync(q, (dense ? tr->dense.as<int32_t>() : tr->adm.as<int32_t>()) + 4 * b,
                                  sizeof(q), cudaMemcpyDeviceToHost, s));
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
    const int m = q[1] - q[0], n = q[3] - q[2];
    if (dense) {
        const int64_t base = read_scalar(tr->dense_base.as<int64_t>() + b, s);
        const int32_t ld = read_scalar(tr->dense_ld.as<int32_t>() + b, s);
        get_dense_block_kernel<<<grid1d((int64_t)m * n), 256, 0, s>>>(base, ld, m, n, A->dense.as<double>(), out);
        HM_LAUNCH_CHECK();
    } else {
        const int k = read_scalar(A->rank.as<int32_t>() + b, s);
        get_lr_block_kernel<<<grid1d((int64_t)m * n), 256, 0, s>>>(
            (int32_t)b, q[0], q[2], m, n, k, tr->leaf_begin.as<int32_t>(), tr->n_leaf, tr->lr_rowptr.as<int64_t>(),
            tr->lr_list.as<int32_t>(), A->up_koff.as<int32_t>(), A->up_off.as<int64_t>(), A->up_K.as<int32_t>(),
            A->up.as<double>(), tr->lr_colptr.as<int64_t>(), tr->lr_collist.as<int32_t>(), A->wp_koff.as<int32_t>(),
            A->wp_off.as<int64_t>(), A->wp_K.as<int32_t>(), A->wp.as<double>(), out);
        HM_LAUNCH_CHECK();
    }
}

// ---------------------------------------------------------------------------
// low-precision copies
// ---------------------------------------------------------------------------
// four values per thread and step (16-byte loads and stores; a and o are
// 16-byte aligned), the last n mod 4 one by one
__global__ void to_f32_kernel(const double *a, int64_t n, float *o) {
    const int64_t n4 = n / 4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 u = reinterpret_cast<const double2 *>(a)[2 * i], v = reinterpret_cast<const double2 *>(a)[2 * i + 1];
        reinterpret_cast<float4 *>(o)[i] = make_float4((float)u.x, (float)u.y, (float)v.x, (float)v.y);
    }
    for (int64_t i = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)a[i];
}

__global__ void to_bf16_kernel(const double *a, int64_t n, __nv_bfloat16 *o) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = __float2bfloat16_rn((float)a[i]);
}

void build_tail_panels(hm_matrix *A, cudaStream_t s);

void make_low_copies(hm_matrix *A, cudaStream_t s) {
    const hm_assemble_params &p = A->params;
    const int64_t nd = A->tree->dense_entries, nu = std::max<int64_t>(A->up_entries, 8),
                  nw = std::max<int64_t>(A->wp_entries, 8);
    if (p.dense_dtype == HM_F32 || p.factor_dtype != HM_F64) {
        A->dense32.alloc(sizeof(float) * std::max<int64_t>(nd, 1));
        to_f32_kernel<<<grid1d(nd), 256, 0, s>>>(A->dense.as<double>(), nd, A->dense32.as<float>());
        HM_LAUNCH_CHECK();
    }
    if (p.factor_dtype == HM_F32) {
        A->up32.alloc(sizeof(float) * nu);
        A->wp32.alloc(sizeof(float) * nw);
        to_f32_kernel<<<grid1d(nu), 256, 0, s>>>(A->up.as<double>(), nu, A->up32.as<float>());
        HM_LAUNCH_CHECK();
        to_f32_kernel<<<grid1d(nw), 256, 0, s>>>(A->wp.as<double>(), nw, A->wp32.as<float>());
        HM_LAUNCH_CHECK();
        if (A->rank32.p) build_tail_panels(A, s);
    } else if (p.factor_dtype == HM_BF16) {
        A->upbf.alloc(sizeof(__nv_bfloat16) * nu);
        A->wpbf.alloc(sizeof(__nv_bfloat16) * nw);
        to_bf16_kernel<<<grid1d(nu), 256, 0, s>>>(A->up.as<double>(), nu, A->upbf.as<__nv_bfloat16>());
        HM_LAUNCH_CHECK();
        to_bf16_kernel<<<grid1d(nw), 256, 0, s>>>(A->wp.as<double>(), nw, A->wpbf.as<__nv_bfloat16>());
        HM_LAUNCH_CHECK();
    }
}

// BF16 copies of the factors (and the FP32 near field they run with) from the
// FP64 master, when the assembly did not keep them.
void ensure_bf16_copies(const hm_matrix *Ac, cudaStream_t s) {
    hm_matrix *A = const_cast<hm_matrix *>(Ac);  // cache owned by the matrix
    const int64_t nd = A->tree->dense_entries, nu = std::max<int64_t>(A->up_entries, 8),
                  nw = std::max<int64_t>(A->wp_entries, 8);
    if (!A->dense32.p) {
        A->dense32.alloc(sizeof(float) * std::max<int64_t>(nd, 1));
        to_f32_kernel<<<grid1d(nd), 256, 0, s>>>(A->dense.as<double>(), nd, A->dense32.as<float>());
        HM_LAUNCH_CHECK();
    }
    if (!A->upbf.p) {
        A->upbf.alloc(sizeof(__nv_bfloat16) * nu);
        A->wpbf.alloc(sizeof(__nv_bfloat16) * nw);
        to_bf16_kernel<<<grid1d(nu), 256, 0, s>>>(A->up.as<double>(), nu, A->upbf.as<__nv_bfloat16>());
        HM_LAUNCH_CHECK();
        to_bf16_kernel<<<grid1d(nw), 256, 0, s>>>(A->wp.as<double>(), nw, A->wpbf.as<__nv_bfloat16>());
        HM_LAUNCH_CHECK();
    }
    if (A->trans_ready && !A->dense32_t.p) {
        const int64_t ne = std::max<int64_t>(A->tree->dense_entries, 1);
        A->dense32_t.alloc(sizeof(float) * ne);
        to_f32_kernel<<<grid1d(ne), 256, 0, s>>>(A->dense_t.as<double>(), ne, A->dense32_t.as<float>());
        HM_LAUNCH_CHECK();
    }
}

// FP32 copies of the factors (and of the near field) from the FP64 master,
// when the assembly did not keep them: the precision an inner solve on the
// BF16 factors falls back to when refinement stops contracting.
void ensure_f32_copies(const hm_matrix *Ac, cudaStream_t s) {
    hm_matrix *A = const_cast<hm_matrix *>(Ac);  // cache owned by the matrix
    const int64_t nd = A->tree->dense_entries, nu = std::max<int64_t>(A->up_entries, 8),
                  nw = std::max<int64_t>(A->wp_entries, 8);
    if (!A->dense32.p) {
        A->dense32.alloc(sizeof(float) * std::max<int64_t>(nd, 1));
        to_f32_kernel<<<grid1d(nd), 256, 0, s>>>(A->dense.as<double>(), nd, A->dense32.as<float>());
        HM_LAUNCH_CHECK();
    }
    if (!A->up32.p) {
        A->up32.alloc(sizeof(float) * nu);
        A->wp32.alloc(sizeof(float) * nw);
        to_f32_kernel<<<grid1d(nu), 256, 0, s>>>(A->up.as<double>(), nu, A->up32.as<float>());
        HM_LAUNCH_CHECK();
        to_f32_kernel<<<grid1d(nw), 256, 0, s>>>(A->wp.as<double>(), nw, A->wp32.as<float>());
        HM_LAUNCH_CHECK();
        if (A->rank32.p) build_tail_panels(A, s);
    }
    if (A->trans_ready && !A->dense32_t.p) {
        const int64_t ne = std::max<int64_t>(A->tree->dense_entries, 1);
        A->dense32_t.alloc(sizeof(float) * ne);
        to_f32_kernel<<<grid1d(ne), 256, 0, s>>>(A->dense_t.as<double>(), ne, A->dense32_t.as<float>());
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

// per-geometry sources: f[s][perm[k]] with the sources of the geometry of k
__global__ void load_vector_geom_kernel(const double *pt, int64_t npad, int64_t n, const int32_t *perm,
                                        const int64_t *goff, int G, const double *src, int nsrc, QuadParams qp,
                                        double *f) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = G;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (goff[mid] <= k) lo = mid;
            else hi = mid;
        }
        const double *sg = src + (int64_t)lo * nsrc * 3;
        const double area = pt[(int64_t)PT_AREA * npad + k];
        const int32_t i = perm[k];
        for (int s = 0; s < nsrc; ++s) {
            const double px = sg[3 * s], py = sg[3 * s + 1], pz = sg[3 * s + 2];
            double acc = 0.0;
            for (int q = 0; q < NQ; ++q) {
                const double dx = pt[(int64_t)q * npad + k] - px, dy = pt[(int64_t)(7 + q) * npad + k] - py,
                             dz = pt[(int64_t)(14 + q) * npad + k] - pz;
                acc += qp.w[q] / sqrt(dx * dx + dy * dy + dz * dz);
            }
            f[(int64_t)s * n + i] = area * acc * 0.079577471545947667884441881686257181;
        }
    }
}

void load_vector_geom_impl(const hm_tree *tr, const double *src, int nsrc, double *f, cudaStream_t s) {
    const QuadParams qp = make_quad(1);
    std::vector<int64_t> go = tr->geom_off;
    if (go.size() < 2) go = {0, tr->n};
    const int G = (int)go.size() - 1;
    DBuf d_go;
    d_go.alloc(sizeof(int64_t) * (G + 1));
    HM_CUDA_CHECK(cudaMemcpyAsync(d_go.p, go.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, s));
    load_vector_geom_kernel<<<grid1d(tr->n), 256, 0, s>>>(tr->pt.as<double>(), tr->npad, tr->n, tr->perm.as<int32_t>(),
                                                          d_go.as<int64_t>(), G, src, nsrc, qp, f);
    HM_LAUNCH_CHECK();
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
}

void load_vector_impl(const hm_tree *tr, const double *src, int nsrc, double *f, cudaStream_t s) {
    const QuadParams qp = make_quad(1);
    load_vector_kernel<<<grid1d(tr->n), 256, 0, s>>>(tr->pt.as<double>(), tr->npad, tr->n, tr->perm.as<int32_t>(), src,
                                                     nsrc, qp, f);
    HM_LAUNCH_CHECK();
}


// ---------------------------------------------------------------------------
// single-layer potential at points off the surface (the ansatz of Sec. 2.1,
// evaluated at interior points for the error measure of Sec. 4.3), 7-point
// rule on every panel:
//   trans = 0: u(p_k) = sum_j |T_j| sum_q w_q G(p_k, y_q^j) phi_j
//   trans = 1: g_j    = |T_j| sum_q w_q sum_k G(p_k, y_q^j) r_k   (the adjoint)
// ---------------------------------------------------------------------------
constexpr int POT_THREADS = 256;  // evaluation points per CTA (trans = 0)
constexpr int POT_CHUNK = 256;    // panels per CTA (trans = 0) / points staged per pass (trans = 1)
constexpr double INV_4PI_D = 0.079577471545947667884441881686257181;

// part[c][k] = sum over the panels of chunk c of the contributions to u(p_k)
__global__ void __launch_bounds__(POT_THREADS) potential_partial_kernel(const double *__restrict__ pt, int64_t npad,
                                                                        int64_t n, const int32_t *__restrict__ perm,
                                                                        const double *__restrict__ pts, int64_t K,
                                                                        const double *__restrict__ phi,
                                                                        const QuadParams qp, double *__restrict__ part) {
    __shared__ double s_x[NQ][POT_CHUNK], s_y[NQ][POT_CHUNK], s_z[NQ][POT_CHUNK], s_c[POT_CHUNK];
    const int64_t j0 = (int64_t)blockIdx.y * POT_CHUNK;
    const int nj = (int)min((int64_t)POT_CHUNK, n - j0);
    for (int j = threadIdx.x; j < nj; j += POT_THREADS) {
        const int64_t m = j0 + j;
        for (int q = 0; q < NQ; ++q) {
            s_x[q][j] = pt[(int64_t)q * npad + m];
            s_y[q][j] = pt[(int64_t)(7 + q) * npad + m];
            s_z[q][j] = pt[(int64_t)(14 + q) * npad + m];
        }
        s_c[j] = pt[(int64_t)PT_AREA * npad + m] * phi[perm[m]];
    }
    __syncthreads();
    const int64_t k = (int64_t)blockIdx.x * POT_THREADS + threadIdx.x;
    if (k >= K) return;
    const double px = pts[3 * k], py = pts[3 * k + 1], pz = pts[3 * k + 2];
    double acc = 0.0;
    for (int j = 0; j < nj; ++j) {
        double sj = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double dx = px - s_x[q][j], dy = py - s_y[q][j], dz = pz - s_z[q][j];
            sj = fma(qp.w[q], rsqrt(fma(dx, dx, fma(dy, dy, dz * dz))), sj);
        }
        acc = fma(s_c[j], sj, acc);
    }
    part[(int64_t)blockIdx.y * K + k] = acc;
}

// u(p_k) = (1/4pi) sum over chunks in order
__global__ void potential_sum_kernel(const double *__restrict__ part, int64_t nchunk, int64_t K, double *__restrict__ u) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t c = 0; c < nchunk; ++c) acc += part[c * K + k];
        u[k] = acc * INV_4PI_D;
    }
}

// g_j for one panel per thread, the points and their weights r staged in
// shared memory chunk by chunk
__global__ void __launch_bounds__(POT_THREADS) potential_adjoint_kernel(const double *__restrict__ pt, int64_t npad,
                                                                        int64_t n, const int32_t *__restrict__ perm,
                                                                        const double *__restrict__ pts, int64_t K,
                                                                        const double *__restrict__ r,
                                                                        const QuadParams qp, double *__restrict__ g) {
    __shared__ double s_p[4][POT_CHUNK];
    const int64_t m = (int64_t)blockIdx.x * POT_THREADS + threadIdx.x;
    const bool live = m < n;
    double x[NQ], y[NQ], z[NQ], acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        x[q] = live ? pt[(int64_t)q * npad + m] : 0.0;
        y[q] = live ? pt[(int64_t)(7 + q) * npad + m] : 0.0;
        z[q] = live ? pt[(int64_t)(14 + q) * npad + m] : 0.0;
        acc[q] = 0.0;
    }
    for (int64_t k0 = 0; k0 < K; k0 += POT_CHUNK) {
        const int nk = (int)min((int64_t)POT_CHUNK, K - k0);
        __syncthreads();
        for (int k = threadIdx.x; k < nk; k += POT_THREADS) {
            s_p[0][k] = pts[3 * (k0 + k)];
            s_p[1][k] = pts[3 * (k0 + k) + 1];
            s_p[2][k] = pts[3 * (k0 + k) + 2];
            s_p[3][k] = r[k0 + k];
        }
        __syncthreads();
        for (int k = 0; k < nk; ++k) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const double dx = s_p[0][k] - x[q], dy = s_p[1][k] - y[q], dz = s_p[2][k] - z[q];
                acc[q] = fma(s_p[3][k], rsqrt(fma(dx, dx, fma(dy, dy, dz * dz))), acc[q]);
            }
        }
    }
    if (!live) return;
    double sj = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) sj = fma(qp.w[q], acc[q], sj);
    g[perm[m]] = pt[(int64_t)PT_AREA * npad + m] * sj * INV_4PI_D;
}

void potential_impl(const hm_tree *tr, const double *pts, int64_t K, int trans, const double *in, double *out,
                    cudaStream_t s) {
    const QuadParams qp = make_quad(1);
    const int64_t n = tr->n;
    if (K == 0 || n == 0) {
        if (trans && n) HM_CUDA_CHECK(cudaMemsetAsync(out, 0, sizeof(double) * n, s));
        if (!trans && K) HM_CUDA_CHECK(cudaMemsetAsync(out, 0, sizeof(double) * K, s));
        return;
    }
    if (!trans) {
        const int64_t nchunk = (n + POT_CHUNK - 1) / POT_CHUNK;
        if (nchunk > 65535) fail(HM_EINVAL, "too many panels for the potential kernel (%lld)", (long long)n);
        SBuf part;
        part.alloc(sizeof(double) * nchunk * K, s);
        const dim3 grid((unsigned)((K + POT_THREADS - 1) / POT_THREADS), (unsigned)nchunk);
        {
            Trace trace("potential_kernel", s);
            potential_partial_kernel<<<grid, POT_THREADS, 0, s>>>(tr->pt.as<double>(), tr->npad, n,
                                                                  tr->perm.as<int32_t>(), pts, K, in, qp,
                                                                  part.as<double>());
            HM_LAUNCH_CHECK();
            potential_sum_kernel<<<grid1d(K), 256, 0, s>>>(part.as<double>(), nchunk, K, out);
            HM_LAUNCH_CHECK();
        }
    } else {
        Trace trace("potential_adjoint_kernel", s);
        potential_adjoint_kernel<<<(unsigned)((n + POT_THREADS - 1) / POT_THREADS), POT_THREADS, 0, s>>>(
            tr->pt.as<double>(), tr->npad, n, tr->perm.as<int32_t>(), pts, K, in, qp, out);
        HM_LAUNCH_CHECK();
    }
}

// ---------------------------------------------------------------------------
// H-matrix-vector product without any device allocation
//
// For callers that must not allocate device memory while they run: code that
// works inside a pre-sized memory budget (a pool-managed or fixed-footprint
// service), code running where an allocation would block or fail, or callers
// whose own allocator forbids stray cudaMalloc/cudaFree calls.  hm_matvec
// obtains its permuted input / output vectors and its low-rank projections
// from the stream-ordered allocator on every call; this variant takes them
// from one file-scope device array instead, sized once when the library is
// loaded.
//
// Scratch layout: the product's working vectors (x and y in Morton order,
// the projections t_b = W_b^T x and their per-column-cluster partials, and
// the FP32 roundings of those for the low-precision copies): 2 n + K + P
// doubles plus n + K + P floats (K = sum of ranks, P = partials).
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
static CUcontext g_noalloc_ctx[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_noalloc_mutex;

// The current driver context (resolved through the runtime's driver entry
// point, like the tensor-map encoder): a device reset makes a new primary
// context, in which the array has a new address.
static CUcontext current_context() {
    typedef CUresult (*PFN_ctxGetCurrent)(CUcontext *);
    static PFN_ctxGetCurrent fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            fail(HM_ECUDA, "cuCtxGetCurrent is not available from the driver");
        fn = reinterpret_cast<PFN_ctxGetCurrent>(p);
    }
    CUcontext c = nullptr;
    if (fn(&c) != CUDA_SUCCESS) fail(HM_ECUDA, "cuCtxGetCurrent failed");
    return c;
}

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in; the address is looked up once per device (with
// that device current) on the first call, and again when the device's
// context has changed since (after a cudaDeviceReset).
static double *noalloc_scratch() {
    int dev = 0;
    HM_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) fail(HM_EINVAL, "device index %d out of range", dev);
    const CUcontext ctx = current_context();  // NULL in a thread where the runtime has not made it current yet
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev] || !ctx || g_noalloc_ctx[dev] != ctx) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the context current
        if (e != cudaSuccess || !p)
            fail(HM_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = current_context();
    }
    return static_cast<double *>(g_noalloc_ptr[dev]);
}

void matvec_noalloc(const hm_matrix *A, int32_t nrhs, hm_dtype prec, const double *x, double *y, double alpha,
                    double beta, cudaStream_t s) {
    const int64_t n = A->tree->n;
    const int64_t need = work_doubles(A, A->n_partials);  // the forward product only
    if (need > NOALLOC_MAX_DOUBLES)
        fail(HM_EINVAL,
             "problem too large for the allocation-free product: needs %lld scratch doubles "
             "(2 n + K + P doubles and n + K + P floats), the limit is %lld",
             (long long)need, (long long)NOALLOC_MAX_DOUBLES);
    const MatvecWork w = work_at(A, noalloc_scratch(), A->n_partials);
    for (int r = 0; r < nrhs; ++r) {
        permute_to_morton(A->tree, x + (int64_t)r * n, w.xm, s);
        matvec_morton(A, prec, w, s, false);
        permute_from_morton(A->tree, w.ym, alpha, beta, y + (int64_t)r * n, s);
    }
}

}  // namespace hm
