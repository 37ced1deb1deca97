// solve.cu -- restarted GMRES and FP64 iterative refinement.
//
// The paper solves the Galerkin system with a hand-written GPU Krylov solver
// (Sec. 4.1; CG to a relative residual of 1e-8).  Here: GMRES(m) in Morton
// order with x_0 = 0; Arnoldi by classical Gram-Schmidt applied twice (CGS2)
// in FP64; Givens rotations, the Hessenberg least-squares problem and the
// triangular solve in FP64 on the device; the Givens estimate ends a cycle and
// the true residual b - H x (FP64 operator) decides convergence.  With
// refinement the inner GMRES applies the FP32 / BF16 copy of H while every
// vector, dot product and rotation stays FP64, and the outer residual uses
// the FP64 master.  Dot products reduce in a fixed order (deterministic).
//
// With use_graph the Arnoldi steps of a cycle run as one CUDA graph: a WHILE
// node whose body is one step (operator, CGS2, Givens) with the step index in
// device memory, and the Givens kernel ends the loop on the device, so the
// host waits once per cycle instead of once per step.  The arithmetic is the
// same kernel for kernel, so both forms give the same iterates.
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <vector>

#include "hm_internal.cuh"

namespace hm {

void matvec_morton(const hm_matrix *A, hm_dtype prec, const MatvecWork &w, cudaStream_t s, bool trans);
void build_transposed(const hm_matrix *A, cudaStream_t s);
int64_t matvec_work_doubles(const hm_matrix *A);
MatvecWork matvec_work_at(const hm_matrix *A, double *base);

// y = op(H) x in Morton order (x and y distinct vectors of the solver); the
// projections live in the solver's workspace
static void apply(const hm_matrix *A, hm_dtype prec, const double *x, double *y, DBuf &work, cudaStream_t s,
                  bool trans) {
    MatvecWork w = matvec_work_at(A, work.as<double>());
    w.xm = const_cast<double *>(x);
    w.ym = y;
    matvec_morton(A, prec, w, s, trans);
}

constexpr int DOT_THREADS = 512;
constexpr int DOT_CHUNK = 8;  // vectors per register pass

// out[l] = V_l . w for l < nv (+ out[l] when accumulate), one launch: every
// block writes its partial sums part[blk][l]; the block that finishes last
// (a ticket counter, reset by it for the next call) adds the partials of
// each l in a fixed order (lanes over blocks, then a fixed shuffle tree).
__global__ void __launch_bounds__(DOT_THREADS) dots_kernel(const double *__restrict__ V, int64_t ld, int nv,
                                                            const double *__restrict__ w, int64_t n,
                                                            double *__restrict__ part, double *__restrict__ out,
                                                            int accumulate, unsigned int *ticket,
                                                            const LoopCtl *ctl) {
    if (ctl) nv = ctl->j + 1;  // graph form: the vectors V_0..V_j of step j
    __shared__ double s[DOT_THREADS / 32][DOT_CHUNK];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(n, i0 + per);
    for (int c0 = 0; c0 < nv; c0 += DOT_CHUNK) {
        double acc[DOT_CHUNK];
#pragma unroll
        for (int c = 0; c < DOT_CHUNK; ++c) acc[c] = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += DOT_THREADS) {
            const double wi = w[i];
#pragma unroll
            for (int c = 0; c < DOT_CHUNK; ++c)
                if (c0 + c < nv) acc[c] = fma(V[(int64_t)(c0 + c) * ld + i], wi, acc[c]);
        }
#pragma unroll
        for (int c = 0; c < DOT_CHUNK; ++c) {
            double v = acc[c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) s[warp][c] = v;
        }
        __syncthreads();
        if (threadIdx.x < DOT_CHUNK && c0 + (int)threadIdx.x < nv) {
            double t = 0.0;
            for (int k = 0; k < DOT_THREADS / 32; ++k) t += s[k][threadIdx.x];
            part[(int64_t)blockIdx.x * nv + c0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int l = warp; l < nv; l += DOT_THREADS / 32) {
        double t = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(part + (int64_t)b * nv + l);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) out[l] = accumulate ? out[l] + t : t;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// w -= sum_l V_l h_l
__global__ void sub_combo_kernel(const double *__restrict__ V, int64_t ld, int nv, const double *__restrict__ h,
                                 int64_t n, double *__restrict__ w, const LoopCtl *ctl) {
    if (ctl) nv = ctl->j + 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = w[i];
        for (int l = 0; l < nv; ++l) acc -= V[(int64_t)l * ld + i] * h[l];
        w[i] = acc;
    }
}

// x += sum_l V_l y_l
__global__ void add_combo_kernel(const double *__restrict__ V, int64_t ld, int nv, const double *__restrict__ y,
                                 int64_t n, double *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < nv; ++l) acc += V[(int64_t)l * ld + i] * y[l];
        x[i] += acc;
    }
}

// dst = src * (1 / norm) where norm = sqrt(*nrm2); dst = src when the norm is 0
__global__ void scale_kernel(const double *src, const double *nrm2, int64_t n, double *dst) {
    const double nr = sqrt(*nrm2);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = nr > 0.0 ? src[i] / nr : 0.0;
}

__global__ void residual_kernel(const double *b, const double *ax, int64_t n, double *r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - ax[i];
}

__global__ void axpy_kernel(double a, const double *x, int64_t n, double *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

// Column j of the Hessenberg matrix (H[l][j], l = 0..j+1, column-major with
// leading dimension m+1): h = first CGS pass + second pass, H[j+1][j] =
// ||w||.  Applies the previous rotations, forms rotation j, updates g, and
// writes |g[j+1]| and H[j+1][j] to est[0], est[1].
__global__ void givens_kernel(double *H, int ldh, int j, const double *h, const double *wn2, double *cs, double *sn,
                              double *g, double *est) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double *col = H + (int64_t)j * ldh;
    for (int l = 0; l <= j; ++l) col[l] = h[l];
    const double hn = sqrt(*wn2);
    col[j + 1] = hn;
    for (int l = 0; l < j; ++l) {
        const double t = cs[l] * col[l] + sn[l] * col[l + 1];
        col[l + 1] = -sn[l] * col[l] + cs[l] * col[l + 1];
        col[l] = t;
    }
    const double rho = hypot(col[j], col[j + 1]);
    cs[j] = rho > 0.0 ? col[j] / rho : 1.0;
    sn[j] = rho > 0.0 ? col[j + 1] / rho : 0.0;
    col[j] = rho;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    est[0] = fabs(g[j + 1]);
    est[1] = hn;
}

// Graph form of one step's bookkeeping (step index j = ctl->j, 0 <= j < m).
// out = V_j
__global__ void vj_copy_kernel(const double *__restrict__ V, int64_t n, int m, const LoopCtl *ctl,
                               double *__restrict__ out) {
    const int j = ctl->j;
    if (j < 0 || j >= m) return;
    const double *src = V + (int64_t)j * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = src[i];
}

// h[l] += y[l], l <= j (the second CGS pass)
__global__ void h_accum_kernel(const double *__restrict__ y, const LoopCtl *ctl, double *__restrict__ h) {
    for (int l = threadIdx.x; l <= ctl->j; l += blockDim.x) h[l] += 1.0 * y[l];
}

// givens_kernel for step j = ctl->j, then the stopping test of the host
// loop (estimate at or below thr, breakdown, or the cycle's step limit):
// ctl->j = j + 1 and the loop's condition is cleared when it stops.  Every
// iteration advances j and j >= lim stops, so the loop ends after at most
// lim <= m iterations.
__global__ void givens_loop_kernel(double *H, int ldh, int m, LoopCtl *ctl, const double *h, const double *wn2,
                                   double *cs, double *sn, double *g, double *est, cudaGraphConditionalHandle loop) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j = ctl->j;
    if (j < 0 || j >= m) {
        cudaGraphSetConditional(loop, 0u);
        return;
    }
    double *col = H + (int64_t)j * ldh;
    for (int l = 0; l <= j; ++l) col[l] = h[l];
    const double hn = sqrt(*wn2);
    col[j + 1] = hn;
    for (int l = 0; l < j; ++l) {
        const double t = cs[l] * col[l] + sn[l] * col[l + 1];
        col[l + 1] = -sn[l] * col[l] + cs[l] * col[l + 1];
        col[l] = t;
    }
    const double rho = hypot(col[j], col[j + 1]);
    cs[j] = rho > 0.0 ? col[j] / rho : 1.0;
    sn[j] = rho > 0.0 ? col[j + 1] / rho : 0.0;
    col[j] = rho;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    est[0] = fabs(g[j + 1]);
    est[1] = hn;
    const int k = j + 1;
    const bool stop = est[0] <= ctl->thr || hn == 0.0 || k >= ctl->lim || k >= m;
    ctl->j = k;
    cudaGraphSetConditional(loop, stop ? 0u : 1u);
}

// V_{j} = w / ||w|| with j = ctl->j (already advanced), j <= m
__global__ void scale_loop_kernel(const double *src, const double *nrm2, int64_t n, int m, const LoopCtl *ctl,
                                  double *V) {
    const int j = ctl->j;
    if (j < 1 || j > m) return;
    const double nr = sqrt(*nrm2);
    double *dst = V + (int64_t)j * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = nr > 0.0 ? src[i] / nr : 0.0;
}

// back substitution R y = g (R = upper k x k of H)
__global__ void trisolve_kernel(const double *H, int ldh, int k, const double *g, double *y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int c = i + 1; c < k; ++c) t -= H[(int64_t)c * ldh + i] * y[c];
        y[i] = t / H[(int64_t)i * ldh + i];
    }
}

__global__ void set_g0_kernel(double *g, const double *nrm2, int m) {
    if (threadIdx.x != 0) return;
    for (int l = 0; l <= m; ++l) g[l] = 0.0;
    g[0] = sqrt(*nrm2);
}

static unsigned g1(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

// ---------------------------------------------------------------------------
// block-Jacobi preconditioner on the leaf clusters' diagonal blocks
// ---------------------------------------------------------------------------
// Blocks of the block-Jacobi preconditioner: runs of consecutive leaf
// clusters (Morton order, never across two geometries) of at most BJ_ROWS
// rows together — five leaf clusters when those have 40 rows, greedily from
// the start of each geometry.  Block b holds the rows
// [bj_begin[b], bj_begin[b+1]) and the leaves [bj_leaf[b], bj_leaf[b+1]).
constexpr int BJ_ROWS = 200;
constexpr int BJ_MAXM = 256;  // largest block (a single leaf may exceed BJ_ROWS)
constexpr int BJ_SMEM_M = 232;  // blocks inverted in shared memory (232^2 floats = 210 KB)

__global__ void bj_size_kernel(const int32_t *begin, int64_t nb, int64_t *sz) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nb; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = begin[r + 1] - begin[r];
        sz[r] = m * m;
    }
}

// D_b = the near-field entries of A(b, b), read from the row panels of the
// leaves of b: the columns whose index falls inside b (the far-field parts
// of the diagonal block are left out)
__global__ void bj_extract_kernel(const int32_t *begin, const int32_t *bleaf, const int32_t *leaf_begin,
                                  const int64_t *rho_off, const int32_t *rho_K, const int64_t *rho_colptr,
                                  const int32_t *colidx, const double *dense, const int64_t *bj_off, double *bj) {
    const int64_t b = blockIdx.x;
    const int32_t b0 = begin[b], m = begin[b + 1] - b0;
    double *D = bj + bj_off[b];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) D[e] = 0.0;
    __syncthreads();
    for (int32_t r = bleaf[b]; r < bleaf[b + 1]; ++r) {
        const int32_t r0 = leaf_begin[r], mr = leaf_begin[r + 1] - r0;
        const int K = rho_K[r];
        const double *P = dense + rho_off[r];
        const int32_t *ci = colidx + rho_colptr[r];
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const int c = ci[k] - b0;
            if (c >= 0 && c < m) {
                // padding columns carry index 0 and value 0: they may alias column 0
                // of the first block only with a zero value, which is skipped
                for (int i = 0; i < mr; ++i) {
                    const double v = P[(int64_t)i * K + k];
                    if (v != 0.0) D[(int64_t)(r0 - b0 + i) * m + c] = v;
                }
            }
        }
    }
}

// In-place Gauss-Jordan inversion of D (diagonally dominant in practice: its
// diagonal holds the self-interactions; no pivoting).
__global__ void bj_invert_kernel(const int32_t *begin, const int64_t *bj_off, double *bj) {
    const int64_t r = blockIdx.x;
    const int m = begin[r + 1] - begin[r];
    if (m <= BJ_SMEM_M) return;  // inverted by bj_invert_smem_kernel
    double *D = bj + bj_off[r];
    __shared__ double s_piv;
    for (int p = 0; p < m; ++p) {
        if (threadIdx.x == 0) {
            double d = D[p * m + p];
            if (!(fabs(d) > 0.0) || !isfinite(d)) d = 1.0;  // empty near-field diagonal (see the FP32 kernel)
            s_piv = 1.0 / d;
            D[p * m + p] = 1.0;
        }
        __syncthreads();
        const double piv = s_piv;
        for (int j = threadIdx.x; j < m; j += blockDim.x) D[p * m + j] *= piv;
        __syncthreads();
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = e / m, j = e - (e / m) * m;
            if (i == p || j == p) continue;
            D[i * m + j] -= D[i * m + p] * D[p * m + j];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            if (i != p) D[i * m + p] = -D[i * m + p] * D[p * m + p];
        __syncthreads();
    }
    // store the inverse transposed (column-major), as bj_apply_kernel reads it
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e - (e / m) * m;
        if (i < j) {
            const double t = D[i * m + j];
            D[i * m + j] = D[j * m + i];
            D[j * m + i] = t;
        }
    }
}

// The same inversion in FP32 with the block in shared memory (blocks of at
// most BJ_SMEM_M rows; the others are left to bj_invert_kernel): the inverse
// only preconditions, the Krylov method and its residuals stay FP64, so an
// FP32-accurate inverse serves the FP64 solve as well as the exact one.
// Writes the FP64 (rounded up from FP32) and FP32 copies, column-major.
constexpr int BJ_INV_THREADS = 512;  // a 32 x 16 grid over the block
__global__ void __launch_bounds__(BJ_INV_THREADS) bj_invert_smem_kernel(const int32_t *begin, const int64_t *bj_off,
                                                                        double *bj, float *bj32) {
    extern __shared__ float s_D[];
    __shared__ float s_row[BJ_SMEM_M], s_col[BJ_SMEM_M];
    __shared__ float s_piv;
    const int64_t r = blockIdx.x;
    const int m = begin[r + 1] - begin[r];
    if (m > BJ_SMEM_M) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double *D = bj + bj_off[r];
    float *D32 = bj32 + bj_off[r];
    for (int e = threadIdx.x; e < m * m; e += BJ_INV_THREADS) s_D[e] = (float)D[e];
    __syncthreads();
    constexpr int NB = (BJ_SMEM_M + 31) / 32;  // columns per thread
    for (int p = 0; p < m; ++p) {
        // pivot, the scaled pivot row and the pivot column, both 0 at p so
        // that the rank-1 update leaves row and column p alone.  A zero (or
        // non-finite) pivot is replaced by 1: a degenerate tree can make a
        // diagonal block admissible (one-panel clusters are at distance 0),
        // leaving its near-field part empty; the preconditioner then acts as
        // the identity there, which right preconditioning tolerates (the
        // residual and the stopping test are those of the unpreconditioned
        // system)
        if (threadIdx.x == 0) {
            float d = s_D[p * m + p];
            if (!(fabsf(d) > 0.0f) || !isfinite(d)) d = s_D[p * m + p] = 1.0f;
            s_piv = 1.0f / d;
        }
        __syncthreads();
        const float piv = s_piv;
        for (int j = threadIdx.x; j < m; j += BJ_INV_THREADS) {
            s_row[j] = j == p ? 0.0f : s_D[p * m + j] * piv;
            s_col[j] = j == p ? 0.0f : s_D[j * m + p];
        }
        __syncthreads();
        float rj[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) rj[b] = tx + 32 * b < m ? s_row[tx + 32 * b] : 0.0f;
        for (int i = ty; i < m; i += BJ_INV_THREADS / 32) {
            const float ci = s_col[i];
            float *Di = s_D + i * m;
#pragma unroll
            for (int b = 0; b < NB; ++b)
                if (tx + 32 * b < m) Di[tx + 32 * b] = fmaf(-ci, rj[b], Di[tx + 32 * b]);
        }
        __syncthreads();
        // the new pivot row and column
        for (int j = threadIdx.x; j < m; j += BJ_INV_THREADS) {
            s_D[p * m + j] = j == p ? piv : s_row[j];
            if (j != p) s_D[j * m + p] = -s_col[j] * piv;
        }
        __syncthreads();
    }
    // column-major (transposed) as bj_apply_kernel reads it
    for (int i = ty; i < m; i += BJ_INV_THREADS / 32)
        for (int j = tx; j < m; j += 32) {
            const float v = s_D[j * m + i];
            D[i * m + j] = (double)v;
            D32[i * m + j] = v;
        }
}

// z_b = D_b^{-1} v_b: one thread per row over the column-major inverse
// (consecutive threads read consecutive rows of one column), v_b staged in
// shared memory; each row sums its columns in order.  trans: z = D^{-T} v,
// the preconditioner of the transposed system (row-major reading).
// TD = double: the FP64 preconditioner; TD = float: its FP32 rounding with
// FP32 accumulation, for the inner solves on the low-precision copies.
// grid.y = column of [cols][n] vectors.
constexpr int BJ_THREADS = 128;
template <class TD>
__global__ void __launch_bounds__(BJ_THREADS) bj_apply_kernel(const int32_t *begin, const int64_t *bj_off,
                                                              const TD *bj, const double *v, double *z, int trans,
                                                              int64_t n) {
    __shared__ TD s_v[BJ_MAXM];
    const int64_t r = blockIdx.x;
    const int32_t r0 = begin[r], m = begin[r + 1] - r0;
    const TD *D = bj + bj_off[r];
    const double *vc = v + (int64_t)blockIdx.y * n;
    double *zc = z + (int64_t)blockIdx.y * n;
    for (int j = threadIdx.x; j < m; j += BJ_THREADS) s_v[j] = (TD)vc[r0 + j];
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += BJ_THREADS) {
        TD acc = 0;
        const int64_t si = trans ? m : 1, sj = trans ? 1 : m;
        for (int j = 0; j < m; ++j) acc = fma(D[j * sj + i * si], s_v[j], acc);
        zc[r0 + i] = (double)acc;
    }
}

// The same for up to BJ_NC columns per CTA (grid.y = column groups): the
// block's inverse is read once for all of them instead of once per column.
// Each column's sum runs over j in the same order as in bj_apply_kernel, so
// the results are the same bit for bit.  The staged columns are laid out
// [j][column] (16-byte loads of 4 or 2 columns) and the 256 threads cover a
// block of up to BJ_MAXM = 256 rows in one pass (measured at level 8, FP32: 0.575 ms
// per 16-column apply with [column][j] and 128 threads).
constexpr int BJ_NC = 16;
constexpr int BJC_THREADS = 256;
template <class TD, class TVec>
__global__ void __launch_bounds__(BJC_THREADS) bj_apply_cols_kernel(const int32_t *begin, const int64_t *bj_off,
                                                                    const TD *bj, const TVec *v, TVec *z,
                                                                    int trans, int64_t n, int cols) {
    __shared__ __align__(16) TD s_v[BJ_MAXM][BJ_NC];
    const int64_t r = blockIdx.x;
    const int32_t r0 = begin[r], m = begin[r + 1] - r0;
    const int c0 = blockIdx.y * BJ_NC, nc = min(BJ_NC, cols - c0);
    const TD *D = bj + bj_off[r];
    for (int e = threadIdx.x; e < BJ_NC * m; e += blockDim.x) {
        const int c = e / m, j = e - c * m;
        s_v[j][c] = c < nc ? (TD)v[(int64_t)(c0 + c) * n + r0 + j] : (TD)0;
    }
    __syncthreads();
    const int64_t si = trans ? m : 1, sj = trans ? 1 : m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        TD acc[BJ_NC];
#pragma unroll
        for (int c = 0; c < BJ_NC; ++c) acc[c] = 0;
#pragma unroll 4
        for (int j = 0; j < m; ++j) {
            const TD d = D[j * sj + i * si];
#pragma unroll
            for (int c = 0; c < BJ_NC; ++c) acc[c] = fma(d, s_v[j][c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < BJ_NC; ++c)
            if (c < nc) z[(int64_t)(c0 + c) * n + r0 + i] = (TVec)acc[c];
    }
}

// threads of a multi-column apply: one per row of the largest block (rounded
// up to a warp), so that no warp of a CTA sits out the product
static unsigned bjc_threads(const hm_matrix *A) {
    const int t = (std::max(A->bj_mmax, 1) + 31) / 32 * 32;
    return (unsigned)std::min(t, BJC_THREADS);
}

__global__ void bj_round_kernel(const double *a, int64_t n, float *o) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)a[i];
}

void bj_setup(const hm_matrix *Ac, cudaStream_t s) {
    hm_matrix *A = const_cast<hm_matrix *>(Ac);  // cache owned by the matrix
    if (A->bj.p) return;
    const hm_tree *tr = A->tree;
    const int64_t nl = tr->n_leaf;
    // the blocks: greedy runs of consecutive leaves of one geometry
    std::vector<int32_t> lb(nl + 1);
    HM_CUDA_CHECK(cudaMemcpyAsync(lb.data(), tr->leaf_begin.p, sizeof(int32_t) * (nl + 1), cudaMemcpyDeviceToHost, s));
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
    std::vector<int64_t> go = tr->geom_off;
    if (go.size() < 2) go = {0, tr->n};
    std::vector<int32_t> begin{0}, bleaf{0};
    size_t g = 0;
    for (int64_t r = 0; r < nl; ++r) {
        while (g + 1 < go.size() && lb[r] >= go[g + 1]) ++g;
        const int32_t cur = begin.back();
        const bool same_geom = cur >= go[g];
        if (r > bleaf.back() && (lb[r + 1] - cur > BJ_ROWS || !same_geom)) {
            begin.push_back(lb[r]);
            bleaf.push_back((int32_t)r);
        }
    }
    begin.push_back((int32_t)tr->n);
    bleaf.push_back((int32_t)nl);
    const int64_t nb = (int64_t)begin.size() - 1;
    A->n_bj = nb;
    A->bj_begin.alloc(sizeof(int32_t) * (nb + 1));
    A->bj_leaf.alloc(sizeof(int32_t) * (nb + 1));
    HM_CUDA_CHECK(cudaMemcpyAsync(A->bj_begin.p, begin.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, s));
    HM_CUDA_CHECK(cudaMemcpyAsync(A->bj_leaf.p, bleaf.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, s));
    A->bj_off.alloc(sizeof(int64_t) * (nb + 1));
    bj_size_kernel<<<g1(nb), 256, 0, s>>>(A->bj_begin.as<int32_t>(), nb, A->bj_off.as<int64_t>());
    HM_LAUNCH_CHECK();
    HM_CUDA_CHECK(cudaMemsetAsync(A->bj_off.as<int64_t>() + nb, 0, sizeof(int64_t), s));
    const int64_t tot = exclusive_scan_i64(A->bj_off.as<int64_t>(), A->bj_off.as<int64_t>(), nb + 1, s);
    DBuf bj;
    bj.alloc(sizeof(double) * std::max<int64_t>(tot, 1));
    {
        Trace trace("bj_extract_kernel", s);
        bj_extract_kernel<<<(unsigned)nb, 256, 0, s>>>(A->bj_begin.as<int32_t>(), A->bj_leaf.as<int32_t>(),
                                                      tr->leaf_begin.as<int32_t>(), tr->rho_off.as<int64_t>(),
                                                      tr->rho_K.as<int32_t>(), tr->rho_colptr.as<int64_t>(),
                                                      tr->colidx.as<int32_t>(), A->dense.as<double>(),
                                                      A->bj_off.as<int64_t>(), bj.as<double>());
        HM_LAUNCH_CHECK();
    }
    A->bj32.alloc(sizeof(float) * std::max<int64_t>(tot, 1));
    int mmax = 0;
    for (int64_t r = 0; r < nb; ++r) mmax = std::max(mmax, begin[r + 1] - begin[r]);
    A->bj_mmax = mmax;
    {
        Trace trace("bj_invert_kernel", s);
        const int msm = std::min(mmax, BJ_SMEM_M);
        const int smem = (int)sizeof(float) * msm * msm;
        HM_CUDA_CHECK(cudaFuncSetAttribute(bj_invert_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        bj_invert_smem_kernel<<<(unsigned)nb, BJ_INV_THREADS, smem, s>>>(A->bj_begin.as<int32_t>(),
                                                                         A->bj_off.as<int64_t>(), bj.as<double>(),
                                                                         A->bj32.as<float>());
        HM_LAUNCH_CHECK();
        if (mmax > BJ_SMEM_M) {
            // wider blocks (single leaves of more than 232 rows): FP64 in global memory
            bj_invert_kernel<<<(unsigned)nb, 256, 0, s>>>(A->bj_begin.as<int32_t>(), A->bj_off.as<int64_t>(),
                                                          bj.as<double>());
            HM_LAUNCH_CHECK();
            bj_round_kernel<<<g1(tot), 256, 0, s>>>(bj.as<double>(), tot, A->bj32.as<float>());
            HM_LAUNCH_CHECK();
        }
    }
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
    A->bj = std::move(bj);
}

// z = M^{-1} v for `cols` vectors [cols][n]; low: the FP32 copy (inner solves)
void bj_apply_cols(const hm_matrix *A, const double *v, double *z, int cols, bool trans, bool low, cudaStream_t s) {
    Trace trace(low ? "bj_apply_kernel.f32" : "bj_apply_kernel", s);
    if (cols > 1) {
        const dim3 grid((unsigned)A->n_bj, (unsigned)((cols + BJ_NC - 1) / BJ_NC));
        if (low)
            bj_apply_cols_kernel<float, double><<<grid, bjc_threads(A), 0, s>>>(
                A->bj_begin.as<int32_t>(), A->bj_off.as<int64_t>(), A->bj32.as<float>(), v, z, trans ? 1 : 0,
                A->tree->n, cols);
        else
            bj_apply_cols_kernel<double, double><<<grid, bjc_threads(A), 0, s>>>(
                A->bj_begin.as<int32_t>(), A->bj_off.as<int64_t>(), A->bj.as<double>(), v, z, trans ? 1 : 0,
                A->tree->n, cols);
        HM_LAUNCH_CHECK();
        return;
    }
    const dim3 grid((unsigned)A->n_bj, (unsigned)cols);
    if (low)
        bj_apply_kernel<float><<<grid, BJ_THREADS, 0, s>>>(A->bj_begin.as<int32_t>(), A->bj_off.as<int64_t>(),
                                                           A->bj32.as<float>(), v, z, trans ? 1 : 0, A->tree->n);
    else
        bj_apply_kernel<double><<<grid, BJ_THREADS, 0, s>>>(A->bj_begin.as<int32_t>(), A->bj_off.as<int64_t>(),
                                                            A->bj.as<double>(), v, z, trans ? 1 : 0, A->tree->n);
    HM_LAUNCH_CHECK();
}

// The FP32 preconditioner on FP32 vectors (the FP32 Krylov vectors of the
// batched inner solves), any number of columns.
void bj_apply_cols_f32(const hm_matrix *A, const float *v, float *z, int cols, cudaStream_t s) {
    Trace trace("bj_apply_kernel.f32", s);
    const dim3 grid((unsigned)A->n_bj, (unsigned)((cols + BJ_NC - 1) / BJ_NC));
    bj_apply_cols_kernel<float, float><<<grid, bjc_threads(A), 0, s>>>(A->bj_begin.as<int32_t>(), A->bj_off.as<int64_t>(),
                                                                   A->bj32.as<float>(), v, z, 0, A->tree->n, cols);
    HM_LAUNCH_CHECK();
}

static void bj_apply(const hm_matrix *A, const double *v, double *z, cudaStream_t s, bool trans, bool low) {
    bj_apply_cols(A, v, z, 1, trans, low, s);
}

struct Gmres {
    int64_t n;
    int m;
    int nblk;
    DBuf V, w, ax, part, h, H, cs, sn, g, y, est, t, nrm, z, d, ticket, ctl, xin;
    std::map<int, std::unique_ptr<LoopGraph>> graphs;  // keyed by precision, preconditioning, transpose
    Gmres(int64_t n_, int m_, int64_t work_doubles, cudaStream_t s) : n(n_), m(m_) {
        // one block per SM: the last block's fixed-order sum over the blocks'
        // partials is the serial part of a dot-product pass (measured best of
        // 1, 2 and 4 blocks per SM with 256 and 512 threads)
        nblk = std::max(1, std::min<int>(num_sms(), (int)((n + 1023) / 1024)));
        V.alloc(sizeof(double) * (int64_t)(m + 1) * n);
        w.alloc(sizeof(double) * n);
        ax.alloc(sizeof(double) * n);
        part.alloc(sizeof(double) * (int64_t)nblk * (m + 1));
        h.alloc(sizeof(double) * (m + 2));
        H.alloc(sizeof(double) * (int64_t)(m + 1) * m);
        cs.alloc(sizeof(double) * m);
        sn.alloc(sizeof(double) * m);
        g.alloc(sizeof(double) * (m + 1));
        y.alloc(sizeof(double) * m);
        est.alloc(sizeof(double) * 2);
        t.alloc(sizeof(double) * work_doubles);
        z.alloc(sizeof(double) * n);
        d.alloc(sizeof(double) * n);
        nrm.alloc(sizeof(double) * 2);
        ticket.alloc(sizeof(unsigned int));
        HM_CUDA_CHECK(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned int), s));
        ctl.alloc(sizeof(LoopCtl));
    }
    // out[0..nv) = V_l . w (accumulate adds to out)
    void dots(const double *Vb, int nv, const double *wv, double *out, int accumulate, cudaStream_t s,
              const LoopCtl *c = nullptr) {
        Trace trace("gmres_dots", s);
        dots_kernel<<<nblk, DOT_THREADS, 0, s>>>(Vb, n, nv, wv, n, part.as<double>(), out, accumulate,
                                                 ticket.as<unsigned int>(), c);
        HM_LAUNCH_CHECK();
    }
    double norm2_host(const double *v, cudaStream_t s) {
        dots(v, 1, v, nrm.as<double>(), 0, s);
        return read_scalar(nrm.as<double>(), s);
    }
};

// Condition estimate sigma_max / sigma_min of the k x k triangular factor R
// of the rotated Hessenberg matrix (column-major, leading dimension ldh):
// H_k = Q R, so R has the singular values of the Arnoldi matrix, which lie
// inside those of the operator (of the preconditioned operator with
// preconditioning).  Power iteration on R^T R for the largest, inverse
// iteration (two triangular solves per step) for the smallest; host FP64.
static double kappa_from_R(const std::vector<double> &H, int ldh, int k) {
    if (k < 1) return 0.0;
    auto R = [&](int i, int j) { return H[(size_t)j * ldh + i]; };
    std::vector<double> v(k, 1.0), w(k), z(k);
    auto normalise = [&](std::vector<double> &a) {
        double t = 0.0;
        for (double x : a) t += x * x;
        t = std::sqrt(t);
        if (t > 0.0)
            for (double &x : a) x /= t;
        return t;
    };
    normalise(v);
    double lmax = 0.0;
    for (int it = 0; it < 40; ++it) {
        for (int i = 0; i < k; ++i) {  // w = R v
            double t = 0.0;
            for (int j = i; j < k; ++j) t += R(i, j) * v[j];
            w[i] = t;
        }
        for (int j = 0; j < k; ++j) {  // z = R^T w
            double t = 0.0;
            for (int i = 0; i <= j; ++i) t += R(i, j) * w[i];
            z[j] = t;
        }
        lmax = normalise(z);
        v = z;
    }
    std::fill(v.begin(), v.end(), 1.0);
    normalise(v);
    double lmin_inv = 0.0;
    for (int it = 0; it < 40; ++it) {
        for (int j = 0; j < k; ++j) {  // R^T w = v (forward)
            double t = v[j];
            for (int i = 0; i < j; ++i) t -= R(i, j) * w[i];
            w[j] = t / R(j, j);
        }
        for (int i = k - 1; i >= 0; --i) {  // R z = w (backward)
            double t = w[i];
            for (int j = i + 1; j < k; ++j) t -= R(i, j) * z[j];
            z[i] = t / R(i, i);
        }
        lmin_inv = normalise(z);
        v = z;
    }
    if (!(lmax > 0.0) || !(lmin_inv > 0.0) || !std::isfinite(lmin_inv)) return 0.0;
    return std::sqrt(lmax * lmin_inv);
}

// The Arnoldi loop of a cycle as a graph: one step per iteration of the
// WHILE node, the step index in G.ctl (the same kernels as the host loop).
static const LoopGraph &step_graph(const hm_matrix *A, hm_dtype prec, Gmres &G, bool precond, bool trans) {
    const int key = (int)prec * 4 + (precond ? 2 : 0) + (trans ? 1 : 0);
    auto it = G.graphs.find(key);
    if (it != G.graphs.end()) return *it->second;
    if (!G.xin.p) G.xin.alloc(sizeof(double) * G.n);
    auto L = std::make_unique<LoopGraph>();
    const int64_t n = G.n;
    const int m = G.m;
    L->build([&](cudaStream_t cs, cudaGraphConditionalHandle loop) {
        double *V = G.V.as<double>(), *w = G.w.as<double>();
        LoopCtl *c = G.ctl.as<LoopCtl>();
        vj_copy_kernel<<<g1(n), 256, 0, cs>>>(V, n, m, c, G.xin.as<double>());
        HM_LAUNCH_CHECK();
        if (precond) {
            bj_apply(A, G.xin.as<double>(), G.z.as<double>(), cs, trans, prec != HM_F64);
            apply(A, prec, G.z.as<double>(), w, G.t, cs, trans);
        } else {
            apply(A, prec, G.xin.as<double>(), w, G.t, cs, trans);
        }
        G.dots(V, 0, w, G.h.as<double>(), 0, cs, c);
        sub_combo_kernel<<<g1(n), 256, 0, cs>>>(V, n, 0, G.h.as<double>(), n, w, c);
        HM_LAUNCH_CHECK();
        G.dots(V, 0, w, G.y.as<double>(), 0, cs, c);
        sub_combo_kernel<<<g1(n), 256, 0, cs>>>(V, n, 0, G.y.as<double>(), n, w, c);
        HM_LAUNCH_CHECK();
        h_accum_kernel<<<1, 128, 0, cs>>>(G.y.as<double>(), c, G.h.as<double>());
        HM_LAUNCH_CHECK();
        G.dots(w, 1, w, G.nrm.as<double>() + 1, 0, cs);
        givens_loop_kernel<<<1, 32, 0, cs>>>(G.H.as<double>(), m + 1, m, c, G.h.as<double>(),
                                             G.nrm.as<double>() + 1, G.cs.as<double>(), G.sn.as<double>(),
                                             G.g.as<double>(), G.est.as<double>(), loop);
        HM_LAUNCH_CHECK();
        scale_loop_kernel<<<g1(n), 256, 0, cs>>>(w, G.nrm.as<double>() + 1, n, m, c, V);
        HM_LAUNCH_CHECK();
    });
    return *(G.graphs[key] = std::move(L));
}

// GMRES(m) for op x = b (Morton order), x in/out.  Returns the status; iters
// and cycles accumulate; relres = final true residual / ||b||.
static hm_status gmres(const hm_matrix *A, hm_dtype prec, const double *b, double *x, double tol, int maxit,
                       Gmres &G, cudaStream_t s, int &iters, int &cycles, double &relres, bool x_is_zero,
                       bool precond, bool trans, bool use_graph, double *kappa = nullptr) {
    const int64_t n = G.n;
    const int m = G.m;
    double *V = G.V.as<double>();
    const double bnorm = std::sqrt(G.norm2_host(b, s));
    if (bnorm == 0.0) {
        HM_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
        relres = 0.0;
        return HM_OK;
    }
    // r0 = b - A x  -> V_0 (unnormalised)
    if (x_is_zero) {
        HM_CUDA_CHECK(cudaMemcpyAsync(V, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    } else {
        apply(A, prec, x, G.ax.as<double>(), G.t, s, trans);
        residual_kernel<<<g1(n), 256, 0, s>>>(b, G.ax.as<double>(), n, V);
        HM_LAUNCH_CHECK();
    }
    double beta = std::sqrt(G.norm2_host(V, s));
    relres = beta / bnorm;
    while (beta > tol * bnorm && iters < maxit) {
        ++cycles;
        G.dots(V, 1, V, G.nrm.as<double>(), 0, s);
        set_g0_kernel<<<1, 32, 0, s>>>(G.g.as<double>(), G.nrm.as<double>(), m);
        HM_LAUNCH_CHECK();
        scale_kernel<<<g1(n), 256, 0, s>>>(V, G.nrm.as<double>(), n, V);
        HM_LAUNCH_CHECK();
        int k = 0;
        if (use_graph) {
            const LoopGraph &L = step_graph(A, prec, G, precond, trans);
            const LoopCtl hc{0, std::min(m, maxit - iters), tol * bnorm};
            HM_CUDA_CHECK(cudaMemcpyAsync(G.ctl.p, &hc, sizeof(hc), cudaMemcpyHostToDevice, s));
            L.launch(s);
            k = read_scalar(&G.ctl.as<LoopCtl>()->j, s);
            L.count(k);
            iters += k;
        }
        for (int j = 0; j < (use_graph ? 0 : m); ++j) {
            double *vj = V + (int64_t)j * n;
            double *w = G.w.as<double>();
            if (precond) {
                // right preconditioning: w = H (M^{-1} v_j)
                bj_apply(A, vj, G.z.as<double>(), s, trans, prec != HM_F64);
                apply(A, prec, G.z.as<double>(), w, G.t, s, trans);
            } else {
                apply(A, prec, vj, w, G.t, s, trans);
            }
            // CGS2
            G.dots(V, j + 1, w, G.h.as<double>(), 0, s);
            {
                Trace trace("gmres_sub_combo", s);
                sub_combo_kernel<<<g1(n), 256, 0, s>>>(V, n, j + 1, G.h.as<double>(), n, w, nullptr);
                HM_LAUNCH_CHECK();
            }
            G.dots(V, j + 1, w, G.y.as<double>(), 0, s);
            {
                Trace trace("gmres_sub_combo", s);
                sub_combo_kernel<<<g1(n), 256, 0, s>>>(V, n, j + 1, G.y.as<double>(), n, w, nullptr);
                HM_LAUNCH_CHECK();
            }
            // h += h2 (second pass coefficients)
            {
                // h[l] += y[l]
                axpy_kernel<<<1, 128, 0, s>>>(1.0, G.y.as<double>(), j + 1, G.h.as<double>());
                HM_LAUNCH_CHECK();
            }
            G.dots(w, 1, w, G.nrm.as<double>() + 1, 0, s);
            givens_kernel<<<1, 32, 0, s>>>(G.H.as<double>(), m + 1, j, G.h.as<double>(), G.nrm.as<double>() + 1,
                                            G.cs.as<double>(), G.sn.as<double>(), G.g.as<double>(),
                                            G.est.as<double>());
            HM_LAUNCH_CHECK();
            double est[2];
            HM_CUDA_CHECK(cudaMemcpyAsync(est, G.est.p, sizeof(est), cudaMemcpyDeviceToHost, s));
            HM_CUDA_CHECK(cudaStreamSynchronize(s));
            ++iters;
            k = j + 1;
            if (est[0] <= tol * bnorm || est[1] == 0.0 || iters >= maxit) break;
            if (j + 1 <= m) {
                scale_kernel<<<g1(n), 256, 0, s>>>(w, G.nrm.as<double>() + 1, n, V + (int64_t)(j + 1) * n);
                HM_LAUNCH_CHECK();
            }
        }
        if (kappa && *kappa == 0.0 && k > 0) {
            // condition estimate from the first cycle's Hessenberg factor
            std::vector<double> Hh((size_t)(m + 1) * k);
            HM_CUDA_CHECK(cudaMemcpyAsync(Hh.data(), G.H.p, sizeof(double) * Hh.size(), cudaMemcpyDeviceToHost, s));
            HM_CUDA_CHECK(cudaStreamSynchronize(s));
            *kappa = kappa_from_R(Hh, m + 1, k);
        }
        trisolve_kernel<<<1, 32, 0, s>>>(G.H.as<double>(), m + 1, k, G.g.as<double>(), G.y.as<double>());
        HM_LAUNCH_CHECK();
        if (precond) {
            // x += M^{-1} (V y)
            HM_CUDA_CHECK(cudaMemsetAsync(G.d.p, 0, sizeof(double) * n, s));
            add_combo_kernel<<<g1(n), 256, 0, s>>>(V, n, k, G.y.as<double>(), n, G.d.as<double>());
            HM_LAUNCH_CHECK();
            bj_apply(A, G.d.as<double>(), G.z.as<double>(), s, trans, prec != HM_F64);
            axpy_kernel<<<g1(n), 256, 0, s>>>(1.0, G.z.as<double>(), n, x);
            HM_LAUNCH_CHECK();
        } else {
            add_combo_kernel<<<g1(n), 256, 0, s>>>(V, n, k, G.y.as<double>(), n, x);
            HM_LAUNCH_CHECK();
        }
        // true residual -> V_0 for the next cycle
        apply(A, prec, x, G.ax.as<double>(), G.t, s, trans);
        residual_kernel<<<g1(n), 256, 0, s>>>(b, G.ax.as<double>(), n, V);
        HM_LAUNCH_CHECK();
        beta = std::sqrt(G.norm2_host(V, s));
        relres = beta / bnorm;
    }
    return beta <= tol * bnorm ? HM_OK : HM_ENOCONV;
}

void permute_to_morton(const hm_tree *tr, const double *x, double *xm, cudaStream_t s);
void permute_from_morton(const hm_tree *tr, const double *ym, double alpha, double beta, double *y, cudaStream_t s);

void ensure_f32_copies(const hm_matrix *A, cudaStream_t s);

// The next inner precision after a refinement step that did not contract:
// BF16 -> FP32 (the FP32 copies are made from the FP64 master if the
// assembly did not keep them); FP32 -> FP64.
hm_dtype raise_inner(const hm_matrix *A, hm_dtype cur, cudaStream_t s) {
    if (cur == HM_BF16) {
        ensure_f32_copies(A, s);
        return HM_F32;
    }
    return HM_F64;
}

hm_status solve_impl(const hm_matrix *A, const double *b_orig, double *x_orig, const hm_solve_params &p,
                     cudaStream_t s, hm_solve_info *info, bool trans) {
    const auto t0 = std::chrono::steady_clock::now();
    const hm_tree *tr = A->tree;
    const int64_t n = tr->n;
    DBuf b, x;
    b.alloc(sizeof(double) * n);
    x.alloc(sizeof(double) * n);
    permute_to_morton(tr, b_orig, b.as<double>(), s);
    HM_CUDA_CHECK(cudaMemsetAsync(x.p, 0, sizeof(double) * n, s));
    Gmres G(n, p.restart, matvec_work_doubles(A), s);
    const bool pc = p.precond == 1;
    if (pc) bj_setup(A, s);
    int iters = 0, cycles = 0, steps = 0;
    double relres = 1.0;
    hm_status st;
    hm_dtype inner_dt = p.refine ? p.inner_dtype : HM_F64;
    double kappa = 0.0;
    if (!p.refine) {
        st = gmres(A, HM_F64, b.as<double>(), x.as<double>(), p.rel_tol, p.max_iter, G, s, iters, cycles, relres, true,
                   pc, trans, p.use_graph != 0, &kappa);
    } else {
        DBuf r, d, ax;
        r.alloc(sizeof(double) * n);
        d.alloc(sizeof(double) * n);
        ax.alloc(sizeof(double) * n);
        HM_CUDA_CHECK(cudaMemcpyAsync(r.p, b.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        const double bnorm = std::sqrt(G.norm2_host(b.as<double>(), s));
        st = HM_ENOCONV;
        relres = 1.0;
        if (bnorm == 0.0) {
            st = HM_OK;
            relres = 0.0;
        }
        const double stall = p.stall_ratio > 0.0 ? p.stall_ratio : 0.5;
        while (st != HM_OK && steps < p.max_refine && iters < p.max_iter) {
            ++steps;
            HM_CUDA_CHECK(cudaMemsetAsync(d.p, 0, sizeof(double) * n, s));
            double inner = 1.0;
            gmres(A, inner_dt, r.as<double>(), d.as<double>(), p.inner_tol, p.max_iter, G, s, iters, cycles, inner,
                  true, pc, trans, p.use_graph != 0, &kappa);
            axpy_kernel<<<g1(n), 256, 0, s>>>(1.0, d.as<double>(), n, x.as<double>());
            HM_LAUNCH_CHECK();
            apply(A, HM_F64, x.as<double>(), ax.as<double>(), G.t, s, trans);
            residual_kernel<<<g1(n), 256, 0, s>>>(b.as<double>(), ax.as<double>(), n, r.as<double>());
            HM_LAUNCH_CHECK();
            const double prev = relres;
            relres = std::sqrt(G.norm2_host(r.as<double>(), s)) / bnorm;
            if (relres <= p.rel_tol) st = HM_OK;
            else if (!(relres <= stall * prev) && inner_dt != HM_F64) inner_dt = raise_inner(A, inner_dt, s);
        }
    }
    permute_from_morton(tr, x.as<double>(), 1.0, 0.0, x_orig, s);
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
    if (info) {
        info->status = st;
        info->iters = iters;
        info->restarts = cycles;
        info->refine_steps = steps;
        info->rel_resid = relres;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->inner_dtype = (int32_t)inner_dt;
        info->kappa_est = kappa;
    }
    return st;
}

}  // namespace hm
