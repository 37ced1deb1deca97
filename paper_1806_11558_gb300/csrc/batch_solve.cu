// batch_solve.cu -- many independent systems solved in lockstep with one
// shared operator application per Arnoldi step.
//
// A system is one right-hand side restricted to one geometry of the tree:
// system s = r * G + g owns the entries [geom_off[g], geom_off[g + 1]) of
// column r of the [R][n] Morton-ordered vectors.  Every system runs its own
// restarted GMRES (CGS2, Givens rotations, Hessenberg solve, all FP64, the
// same algorithm as solve.cu), but the systems advance together, so one
// step applies H to all R columns at once: on the FP32 / BF16 copies that is
// the 16-right-hand-side tensor-core product of mrhs.cu; on the FP64 master
// it is one product per column.  A system that has converged stops updating
// (its rotations, coefficients and vectors are left alone) while the others
// continue.  The FP64 iterative refinement around it follows solve.cu: the
// residual B - H_64 X in FP64, the inner solves on the low-precision copy.
// Every reduction runs in a fixed order.  With use_graph the lockstep
// Arnoldi steps of a cycle run as one CUDA graph (a WHILE node over one step,
// the per-system stops and the end of the loop decided on the device).
#include <chrono>
#include <cmath>
#include <map>
#include <memory>

#include "hm_internal.cuh"

namespace hm {

void matvec_morton(const hm_matrix *A, hm_dtype prec, const MatvecWork &w, cudaStream_t s, bool trans);
int64_t matvec_work_doubles(const hm_matrix *A);
MatvecWork matvec_work_at(const hm_matrix *A, double *base);
void matvec_mrhs_cols(const hm_matrix *A, hm_dtype prec, const void *x, bool x_f32, int nr, double *Y, void *out,
                      bool out_f32, float *work, cudaStream_t s);
int64_t mrhs_work_floats(const hm_matrix *A);
void mrhs_prepare(const hm_matrix *A, hm_dtype prec, cudaStream_t s);
void bj_setup(const hm_matrix *A, cudaStream_t s);
void bj_apply_cols(const hm_matrix *A, const double *v, double *z, int cols, bool trans, bool low, cudaStream_t s);
void bj_apply_cols_f32(const hm_matrix *A, const float *v, float *z, int cols, cudaStream_t s);
void permute_to_morton(const hm_tree *tr, const double *x, double *xm, cudaStream_t s);
void permute_from_morton(const hm_tree *tr, const double *ym, double alpha, double beta, double *y, cudaStream_t s);
hm_dtype raise_inner(const hm_matrix *A, hm_dtype cur, cudaStream_t s);
int mrhs_error(const hm_matrix *A, cudaStream_t s);
int64_t df_work_floats(const hm_matrix *A);
void matvec_df_morton(const hm_matrix *A, const double *xv, int nr, double *yv, float *work, cudaStream_t s);

constexpr int BMR = 16;        // columns of one tensor-core product
constexpr int BITEM = 8192;    // entries of one work item
constexpr int BTHREADS = 256;

struct Item {
    int32_t sys, col;
    int64_t i0, i1;
};

static unsigned gx(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 65535)); }

// part[item][l] = V_l(col, i0:i1) . w(col, i0:i1), l < nv (0 for inactive systems).
// Warp k of the CTA takes the k-th contiguous chunk of the item and runs over
// the vectors, eight (FP64: four) per pass over the chunk (the chunk of w is
// loaded once per pass): per vector its lanes stride the chunk with four
// independent accumulators and add them by shuffles (the same elements in the
// same order whether a vector is taken in a pass or alone); the eight warps'
// sums of each vector are added in a fixed order at the end, so the CTA
// synchronises once.  TV: the type of the Krylov vectors and of the
// arithmetic up to the warp sums (FP64; FP32 for the FP32 Krylov vectors of
// the inner solves), FP64 from there on.
constexpr int BMAXV = 129;  // restart + 1
template <class TV>
__global__ void __launch_bounds__(BTHREADS) bdots_kernel(const Item *__restrict__ items, const TV *__restrict__ V,
                                                         int64_t vstride, int64_t n, int nv,
                                                         const TV *__restrict__ w, const int *__restrict__ act,
                                                         double *__restrict__ part, const LoopCtl *ctl) {
    if (ctl) nv = ctl->j + 1;
    constexpr int BW = BTHREADS / 32, NQ = sizeof(TV) == 4 ? 8 : 4;
    __shared__ double s_part[BW][BMAXV];
    const Item it = items[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool on = act[it.sys] != 0;
    const int64_t len = it.i1 - it.i0;
    const int64_t chunk = ((len + BW - 1) / BW + 31) / 32 * 32;
    const int64_t c0 = it.i0 + warp * chunk, c1 = min(it.i1, c0 + chunk);
    const TV *wc = w + (int64_t)it.col * n;
    const TV *vb = V + (int64_t)it.col * n;
    int l = 0;
    for (; l + NQ <= nv; l += NQ) {
        TV a[NQ][4];
#pragma unroll
        for (int q = 0; q < NQ; ++q) a[q][0] = a[q][1] = a[q][2] = a[q][3] = 0;
        if (on) {
            const TV *v0 = vb + (int64_t)l * vstride;
            int64_t i = c0 + lane;
            for (; i + 96 < c1; i += 128) {
                const TV w0 = wc[i], w1 = wc[i + 32], w2 = wc[i + 64], w3 = wc[i + 96];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const TV *vq = v0 + q * vstride;
                    a[q][0] = fma(vq[i], w0, a[q][0]);
                    a[q][1] = fma(vq[i + 32], w1, a[q][1]);
                    a[q][2] = fma(vq[i + 64], w2, a[q][2]);
                    a[q][3] = fma(vq[i + 96], w3, a[q][3]);
                }
            }
            for (; i < c1; i += 32) {
                const TV w0 = wc[i];
#pragma unroll
                for (int q = 0; q < NQ; ++q) a[q][0] = fma(v0[q * vstride + i], w0, a[q][0]);
            }
        }
        TV t[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) t[q] = (a[q][0] + a[q][1]) + (a[q][2] + a[q][3]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < NQ; ++q) t[q] += __shfl_xor_sync(0xffffffffu, t[q], o);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < NQ; ++q) s_part[warp][l + q] = (double)t[q];
    }
    for (; l < nv; ++l) {
        TV a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        if (on) {
            const TV *vl = vb + (int64_t)l * vstride;
            int64_t i = c0 + lane;
            for (; i + 96 < c1; i += 128) {
                a0 = fma(vl[i], wc[i], a0);
                a1 = fma(vl[i + 32], wc[i + 32], a1);
                a2 = fma(vl[i + 64], wc[i + 64], a2);
                a3 = fma(vl[i + 96], wc[i + 96], a3);
            }
            for (; i < c1; i += 32) a0 = fma(vl[i], wc[i], a0);
        }
        TV t = (a0 + a1) + (a2 + a3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_part[warp][l] = (double)t;
    }
    __syncthreads();
    for (int l2 = threadIdx.x; l2 < nv; l2 += BTHREADS) {
        double t = 0.0;
        for (int k = 0; k < BW; ++k) t += s_part[k][l2];
        part[(int64_t)blockIdx.x * nv + l2] = t;
    }
}

// out[s][l] = sum over the items of s (in order) of part[item][l]; accumulate adds
__global__ void bdots_final_kernel(const int64_t *__restrict__ iptr, int S, int nv, const double *__restrict__ part,
                                   double *__restrict__ out, int ld, int accumulate, const LoopCtl *ctl) {
    if (ctl) nv = ctl->j + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S * nv; e += gridDim.x * blockDim.x) {
        const int s = e / nv, l = e - (e / nv) * nv;
        double t = 0.0;
        // eight partials' loads in flight, added in item order
#pragma unroll 8
        for (int64_t k = iptr[s]; k < iptr[s + 1]; ++k) t += part[k * nv + l];
        out[(int64_t)s * ld + l] = accumulate ? out[(int64_t)s * ld + l] + t : t;
    }
}

// w(col, i) -= sum_l V_l(col, i) h[s][l]   (active systems; h rounded to TV)
template <class TV>
__global__ void bsub_kernel(const Item *__restrict__ items, const TV *__restrict__ V, int64_t vstride, int64_t n,
                            int nv, const double *__restrict__ h, int ldh, const int *__restrict__ act,
                            TV *__restrict__ w, const LoopCtl *ctl) {
    __shared__ TV s_h[BMAXV];
    if (ctl) nv = ctl->j + 1;
    const Item it = items[blockIdx.x];
    if (!act[it.sys]) return;
    const double *hs = h + (int64_t)it.sys * ldh;
    for (int l = threadIdx.x; l < nv; l += blockDim.x) s_h[l] = (TV)hs[l];
    __syncthreads();
    TV *wc = w + (int64_t)it.col * n;
    constexpr int EPT = BITEM / 256;  // elements per thread of a full item
    if (blockDim.x == 256 && it.i1 - it.i0 == BITEM) {
        // the thread's elements in registers, the vectors one after the other:
        // EPT loads in flight per vector, each element's sum in the same order
        const TV *vb = V + (int64_t)it.col * n + it.i0 + threadIdx.x;
        TV a[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) a[q] = wc[it.i0 + threadIdx.x + 256 * q];
        for (int l = 0; l < nv; ++l) {
            const TV *vl = vb + (int64_t)l * vstride;
            const TV hl = s_h[l];
#pragma unroll
            for (int q = 0; q < EPT; ++q) a[q] -= vl[256 * q] * hl;
        }
#pragma unroll
        for (int q = 0; q < EPT; ++q) wc[it.i0 + threadIdx.x + 256 * q] = a[q];
        return;
    }
    for (int64_t i = it.i0 + threadIdx.x; i < it.i1; i += blockDim.x) {
        TV a = wc[i];
        // eight vectors' loads in flight (the sum order is unchanged; 16 deep
        // measured 0.60 ms against 0.51 ms at level 8)
#pragma unroll 8
        for (int l = 0; l < nv; ++l) a -= V[(int64_t)l * vstride + (int64_t)it.col * n + i] * s_h[l];
        wc[i] = a;
    }
}

// x(col, i) += sum_{l < k_s} V_l(col, i) y[s][l]   (the sum in TV, y rounded to TV)
template <class TV>
__global__ void badd_kernel(const Item *__restrict__ items, const TV *__restrict__ V, int64_t vstride, int64_t n,
                            const int *__restrict__ k, const double *__restrict__ y, int ldy, double *__restrict__ x) {
    __shared__ TV s_y[BMAXV];
    const Item it = items[blockIdx.x];
    const int ks = k[it.sys];
    if (ks == 0) return;
    const double *ys = y + (int64_t)it.sys * ldy;
    for (int l = threadIdx.x; l < ks; l += blockDim.x) s_y[l] = (TV)ys[l];
    __syncthreads();
    double *xc = x + (int64_t)it.col * n;
    for (int64_t i = it.i0 + threadIdx.x; i < it.i1; i += blockDim.x) {
        TV a = 0;
#pragma unroll 8
        for (int l = 0; l < ks; ++l) a += V[(int64_t)l * vstride + (int64_t)it.col * n + i] * s_y[l];
        xc[i] += (double)a;
    }
}

// dst(col, i) = src(col, i) / sqrt(nrm2[s]) for the systems in mask (0 when
// the norm is 0); FP32 vectors are multiplied by the rounded reciprocal
template <class TV>
__global__ void bscale_kernel(const Item *__restrict__ items, const TV *__restrict__ src, int64_t n,
                              const double *__restrict__ nrm2, int nstride, const int *__restrict__ mask,
                              TV *__restrict__ dst, const LoopCtl *ctl, int64_t vs, int m) {
    if (ctl) {
        // graph form: dst = V_j with j = ctl->j (already advanced), 1 <= j <= m
        const int j = ctl->j;
        if (j < 1 || j > m) return;
        dst += (int64_t)j * vs;
    }
    const Item it = items[blockIdx.x];
    if (!mask[it.sys]) return;
    const double nr = sqrt(nrm2[(int64_t)it.sys * nstride]);
    const TV *sc = src + (int64_t)it.col * n;
    TV *dc = dst + (int64_t)it.col * n;
    if (sizeof(TV) == 8) {
        for (int64_t i = it.i0 + threadIdx.x; i < it.i1; i += blockDim.x) dc[i] = nr > 0.0 ? (TV)(sc[i] / nr) : (TV)0;
    } else {
        const TV rinv = nr > 0.0 ? (TV)(1.0 / nr) : (TV)0;
        for (int64_t i = it.i0 + threadIdx.x; i < it.i1; i += blockDim.x) dc[i] = sc[i] * rinv;
    }
}

// out = a - b (rounded to TO)
template <class TO>
__global__ void bsub_vec_kernel(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                                TO *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (TO)(a[i] - b[i]);
}

// out = a rounded to FP32
__global__ void round_vec_kernel(const double *__restrict__ a, int64_t n, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)a[i];
}

__global__ void badd_vec_kernel(const double *__restrict__ a, int64_t n, double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] += a[i];
}

// h[s][l] += h2[s][l], l < nv
__global__ void badd_coef_kernel(int S, int nv, int ld, const double *__restrict__ h2, double *__restrict__ h,
                                 const LoopCtl *ctl) {
    if (ctl) nv = ctl->j + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S * nv; e += gridDim.x * blockDim.x) {
        const int s = e / nv, l = e - (e / nv) * nv;
        h[(int64_t)s * ld + l] += h2[(int64_t)s * ld + l];
    }
}

// Givens step j of every active system (one thread per system); writes
// est[s] = |g_s[j+1]| and hn[s] = ||w_s||
__global__ void bgivens_kernel(int S, int m, int j, int *__restrict__ act, const double *__restrict__ h,
                               int ldh, const double *__restrict__ wn2, double *__restrict__ H,
                               double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ g,
                               double *__restrict__ est, double *__restrict__ hn, const LoopCtl *ctl,
                               const double *__restrict__ thr, int *__restrict__ kk) {
    if (ctl) j = ctl->j;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || !act[s] || j < 0 || j >= m) return;
    double *col = H + (int64_t)s * (m + 1) * m + (int64_t)j * (m + 1);
    double *c = cs + (int64_t)s * m, *sg = sn + (int64_t)s * m, *gs = g + (int64_t)s * (m + 1);
    for (int l = 0; l <= j; ++l) col[l] = h[(int64_t)s * ldh + l];
    const double hh = sqrt(wn2[s]);
    col[j + 1] = hh;
    for (int l = 0; l < j; ++l) {
        const double t = c[l] * col[l] + sg[l] * col[l + 1];
        col[l + 1] = -sg[l] * col[l] + c[l] * col[l + 1];
        col[l] = t;
    }
    const double rho = hypot(col[j], col[j + 1]);
    c[j] = rho > 0.0 ? col[j] / rho : 1.0;
    sg[j] = rho > 0.0 ? col[j + 1] / rho : 0.0;
    col[j] = rho;
    col[j + 1] = 0.0;
    gs[j + 1] = -sg[j] * gs[j];
    gs[j] = c[j] * gs[j];
    est[s] = fabs(gs[j + 1]);
    hn[s] = hh;
    if (ctl) {
        // graph form: the per-system stopping test of the host loop
        kk[s] = j + 1;
        if (est[s] <= thr[s] || hh == 0.0 || j + 1 >= ctl->lim) act[s] = 0;
    }
}

// Graph form, end of step j: advance ctl->j and end the loop when no system
// is active or the cycle's step limit is reached (j grows every iteration and
// j >= lim stops, so the loop ends after at most lim <= m iterations).
__global__ void bstep_end_kernel(int S, int m, const int *__restrict__ act, LoopCtl *ctl,
                                 cudaGraphConditionalHandle loop) {
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    int any = 0;
    for (int k = threadIdx.x; k < S; k += blockDim.x) any |= act[k];
    if (any) atomicOr(&s_any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int k = ctl->j + 1;
        ctl->j = k;
        cudaGraphSetConditional(loop, (s_any && k < ctl->lim && k < m) ? 1u : 0u);
    }
}

// out = V_j (all columns) with j = ctl->j
template <class TV>
__global__ void bvj_copy_kernel(const TV *__restrict__ V, int64_t vs, int m, const LoopCtl *ctl,
                                TV *__restrict__ out) {
    const int j = ctl->j;
    if (j < 0 || j >= m) return;
    const TV *src = V + (int64_t)j * vs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < vs; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = src[i];
}

// y_s = R_s^{-1} g_s over the k_s first rotations (one thread per system)
__global__ void btrisolve_kernel(int S, int m, const int *__restrict__ k, const double *__restrict__ H,
                                 const double *__restrict__ g, double *__restrict__ y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int ks = k[s];
    const double *Hs = H + (int64_t)s * (m + 1) * m;
    const double *gs = g + (int64_t)s * (m + 1);
    double *ys = y + (int64_t)s * m;
    for (int i = ks - 1; i >= 0; --i) {
        double t = gs[i];
        for (int c = i + 1; c < ks; ++c) t -= Hs[(int64_t)c * (m + 1) + i] * ys[c];
        ys[i] = t / Hs[(int64_t)i * (m + 1) + i];
    }
}

// g_s = (sqrt(nrm2[s]), 0, ...) for the systems in mask
__global__ void bset_g0_kernel(int S, int m, const int *__restrict__ mask, const double *__restrict__ nrm2,
                               double *__restrict__ g) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S || !mask[s]) return;
    double *gs = g + (int64_t)s * (m + 1);
    for (int l = 0; l <= m; ++l) gs[l] = 0.0;
    gs[0] = sqrt(nrm2[s]);
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
struct Batch {
    const hm_matrix *A;
    int64_t n;
    int R, G, S, m;
    bool precond;
    std::vector<Item> items_h;
    std::vector<int64_t> iptr_h;
    DBuf items, iptr, V, W, Z, AX, part, h, h2, H, cs, sn, g, y, est, hn, nrm, act, cyc, kk, ones, mv, mvf, ctl, thr, xin;
    // FP32 Krylov vectors of the inner solves on the low-precision copies
    // (more than one right-hand side): basis, new vector, preconditioned vector
    DBuf V32, W32, Z32, xin32;
    bool v32 = false;
    int64_t vstride;
    std::map<int, std::unique_ptr<LoopGraph>> graphs;  // graph form of the Arnoldi loop, keyed by precision

    Batch(const hm_matrix *A_, int R_, int m_, bool pc, hm_dtype inner, cudaStream_t s)
        : A(A_), R(R_), m(m_), precond(pc) {
        const hm_tree *tr = A->tree;
        n = tr->n;
        std::vector<int64_t> go = tr->geom_off;
        if (go.size() < 2) go = {0, n};
        G = (int)go.size() - 1;
        S = R * G;
        iptr_h.assign(S + 1, 0);
        for (int r = 0; r < R; ++r)
            for (int gg = 0; gg < G; ++gg) {
                const int sys = r * G + gg;
                iptr_h[sys] = (int64_t)items_h.size();
                for (int64_t i0 = go[gg]; i0 < go[gg + 1]; i0 += BITEM)
                    items_h.push_back(Item{sys, r, i0, std::min<int64_t>(go[gg + 1], i0 + BITEM)});
            }
        iptr_h[S] = (int64_t)items_h.size();
        items.alloc(sizeof(Item) * std::max<size_t>(items_h.size(), 1));
        iptr.alloc(sizeof(int64_t) * (S + 1));
        HM_CUDA_CHECK(cudaMemcpyAsync(items.p, items_h.data(), sizeof(Item) * items_h.size(), cudaMemcpyHostToDevice, s));
        HM_CUDA_CHECK(cudaMemcpyAsync(iptr.p, iptr_h.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, s));
        vstride = (int64_t)R * n;
        W.alloc(sizeof(double) * vstride);
        Z.alloc(sizeof(double) * vstride);
        v32 = R > 1 && inner != HM_F64;
        AX.alloc(sizeof(double) * vstride);
        part.alloc(sizeof(double) * std::max<size_t>(items_h.size(), 1) * (m + 1));
        h.alloc(sizeof(double) * S * (m + 1));
        h2.alloc(sizeof(double) * S * (m + 1));
        H.alloc(sizeof(double) * S * (int64_t)(m + 1) * m);
        cs.alloc(sizeof(double) * S * m);
        sn.alloc(sizeof(double) * S * m);
        g.alloc(sizeof(double) * S * (m + 1));
        y.alloc(sizeof(double) * S * m);
        est.alloc(sizeof(double) * S);
        hn.alloc(sizeof(double) * S);
        nrm.alloc(sizeof(double) * S);
        act.alloc(sizeof(int) * S);
        cyc.alloc(sizeof(int) * S);
        kk.alloc(sizeof(int) * S);
        ones.alloc(sizeof(int) * S);
        ctl.alloc(sizeof(LoopCtl));
        thr.alloc(sizeof(double) * S);
        {
            std::vector<int> o(S, 1);
            HM_CUDA_CHECK(cudaMemcpyAsync(ones.p, o.data(), sizeof(int) * S, cudaMemcpyHostToDevice, s));
            HM_CUDA_CHECK(cudaStreamSynchronize(s));
        }
        mv.alloc(sizeof(double) * matvec_work_doubles(A));
        if (R > 1 && inner != HM_F64) {
            mrhs_prepare(A, inner, s);
            mvf.alloc(sizeof(float) * mrhs_work_floats(A));
        }
    }
    unsigned nitems() const { return (unsigned)items_h.size(); }

    // the Krylov basis in TV ([m + 1][R][n], Morton), allocated and zeroed on first use
    template <class TV> TV *basis(cudaStream_t s) {
        DBuf &b = sizeof(TV) == 4 ? V32 : V;
        if (!b.p) {
            b.alloc(sizeof(TV) * (int64_t)(m + 1) * vstride);
            HM_CUDA_CHECK(cudaMemsetAsync(b.p, 0, sizeof(TV) * (int64_t)(m + 1) * vstride, s));
        }
        return b.as<TV>();
    }
    // the new Arnoldi vector and its preconditioned input in TV
    template <class TV> TV *wvec() {
        if (sizeof(TV) == 8) return W.as<TV>();
        if (!W32.p) W32.alloc(sizeof(float) * vstride);
        return W32.as<TV>();
    }
    template <class TV> TV *zvec() {
        if (sizeof(TV) == 8) return Z.as<TV>();
        if (!Z32.p) Z32.alloc(sizeof(float) * vstride);
        return Z32.as<TV>();
    }

    // outer residual products by the double-float 16-column product (resid_df)
    DBuf dfw;
    void enable_df() { dfw.alloc(sizeof(float) * df_work_floats(A)); }
    // y = H_64 x for all R columns ([R][n], Morton): the outer products of the refinement
    void apply_outer(const double *x, double *yv, cudaStream_t s) {
        if (!dfw.p) {
            apply(HM_F64, x, yv, s);
            return;
        }
        for (int r0 = 0; r0 < R; r0 += BMR)
            matvec_df_morton(A, x + (int64_t)r0 * n, std::min(BMR, R - r0), yv + (int64_t)r0 * n, dfw.as<float>(), s);
    }

    // out[s][l] = V_l . w per system, l < nv
    template <class TV>
    void dots(const TV *Vb, int nv, const TV *w, const int *mask, double *out, int ld, int accumulate,
              cudaStream_t s, const LoopCtl *c = nullptr) {
        Trace trace("batch_dots", s);
        bdots_kernel<TV><<<nitems(), BTHREADS, 0, s>>>(items.as<Item>(), Vb, vstride, n, nv, w, mask,
                                                       part.as<double>(), c);
        HM_LAUNCH_CHECK();
        bdots_final_kernel<<<gx((int64_t)S * (c ? m : nv)), 256, 0, s>>>(iptr.as<int64_t>(), S, nv, part.as<double>(),
                                                                        out, ld, accumulate, c);
        HM_LAUNCH_CHECK();
    }
    // per-system squared norms of v into nrm (host copy returned)
    template <class TV> std::vector<double> norms2(const TV *v, cudaStream_t s) {
        dots(v, 1, v, ones.as<int>(), nrm.as<double>(), 1, 0, s);
        std::vector<double> out(S);
        HM_CUDA_CHECK(cudaMemcpyAsync(out.data(), nrm.p, sizeof(double) * S, cudaMemcpyDeviceToHost, s));
        HM_CUDA_CHECK(cudaStreamSynchronize(s));
        return out;
    }
    // y = op x for all R columns ([R][n], Morton); FP32 vectors (TI / TO =
    // float) only with the low-precision copies and R > 1
    template <class TI, class TO> void apply(hm_dtype prec, const TI *x, TO *yv, cudaStream_t s) {
        if (prec == HM_F64 || R == 1) {
            if (sizeof(TI) != 8 || sizeof(TO) != 8) fail(HM_EINTERNAL, "FP32 Krylov vectors need the block product");
            for (int r = 0; r < R; ++r) {
                MatvecWork w = matvec_work_at(A, mv.as<double>());
                w.xm = reinterpret_cast<double *>(const_cast<TI *>(x + (int64_t)r * n));
                w.ym = reinterpret_cast<double *>(yv + (int64_t)r * n);
                matvec_morton(A, prec, w, s, false);
            }
            return;
        }
        // the workspace of the 16-column product: [n][16] FP32 (unused here), Y, then its work
        float *X = mvf.as<float>();
        double *Y = reinterpret_cast<double *>(X + (int64_t)BMR * n);
        float *work = X + 3 * (int64_t)BMR * n;
        for (int r0 = 0; r0 < R; r0 += BMR) {
            const int nr = std::min(BMR, R - r0);
            matvec_mrhs_cols(A, prec, x + (int64_t)r0 * n, sizeof(TI) == 4, nr, Y, yv + (int64_t)r0 * n,
                             sizeof(TO) == 4, work, s);
        }
    }
    void bj(const double *v, double *z, bool low, cudaStream_t s) { bj_apply_cols(A, v, z, R, false, low, s); }
    void bj(const float *v, float *z, bool, cudaStream_t s) { bj_apply_cols_f32(A, v, z, R, s); }
};

// The lockstep Arnoldi loop of a cycle as a graph: one step per iteration of
// the WHILE node, the step index in B.ctl (the same kernels as the host loop).
template <class TV> static const LoopGraph &batch_step_graph(Batch &B, hm_dtype prec, cudaStream_t s) {
    auto it = B.graphs.find((int)prec);
    if (it != B.graphs.end()) return *it->second;
    const int S = B.S, m = B.m;
    const int64_t vs = B.vstride;
    DBuf &xb = sizeof(TV) == 4 ? B.xin32 : B.xin;
    if (!xb.p) xb.alloc(sizeof(TV) * vs);
    TV *V = B.basis<TV>(s), *w = B.wvec<TV>(), *xin = xb.as<TV>(), *z = B.zvec<TV>();
    auto L = std::make_unique<LoopGraph>();
    L->build([&](cudaStream_t cs, cudaGraphConditionalHandle loop) {
        LoopCtl *c = B.ctl.as<LoopCtl>();
        bvj_copy_kernel<TV><<<gx(vs), 256, 0, cs>>>(V, vs, m, c, xin);
        HM_LAUNCH_CHECK();
        if (B.precond) {
            B.bj(xin, z, prec != HM_F64, cs);
            B.apply(prec, z, w, cs);
        } else {
            B.apply(prec, xin, w, cs);
        }
        B.dots(V, 0, w, B.cyc.as<int>(), B.h.as<double>(), m + 1, 0, cs, c);
        bsub_kernel<TV><<<B.nitems(), 256, 0, cs>>>(B.items.as<Item>(), V, vs, B.n, 0, B.h.as<double>(), m + 1,
                                                    B.cyc.as<int>(), w, c);
        HM_LAUNCH_CHECK();
        B.dots(V, 0, w, B.cyc.as<int>(), B.h2.as<double>(), m + 1, 0, cs, c);
        bsub_kernel<TV><<<B.nitems(), 256, 0, cs>>>(B.items.as<Item>(), V, vs, B.n, 0, B.h2.as<double>(), m + 1,
                                                    B.cyc.as<int>(), w, c);
        HM_LAUNCH_CHECK();
        badd_coef_kernel<<<gx((int64_t)S * m), 256, 0, cs>>>(S, 0, m + 1, B.h2.as<double>(), B.h.as<double>(), c);
        HM_LAUNCH_CHECK();
        B.dots(w, 1, w, B.cyc.as<int>(), B.nrm.as<double>(), 1, 0, cs);
        bgivens_kernel<<<(S + 127) / 128, 128, 0, cs>>>(S, m, 0, B.cyc.as<int>(), B.h.as<double>(), m + 1,
                                                       B.nrm.as<double>(), B.H.as<double>(), B.cs.as<double>(),
                                                       B.sn.as<double>(), B.g.as<double>(), B.est.as<double>(),
                                                       B.hn.as<double>(), c, B.thr.as<double>(), B.kk.as<int>());
        HM_LAUNCH_CHECK();
        bstep_end_kernel<<<1, 256, 0, cs>>>(S, m, B.cyc.as<int>(), c, loop);
        HM_LAUNCH_CHECK();
        bscale_kernel<TV><<<B.nitems(), 256, 0, cs>>>(B.items.as<Item>(), w, B.n, B.nrm.as<double>(), 1,
                                                      B.cyc.as<int>(), V, c, vs, m);
        HM_LAUNCH_CHECK();
    });
    return *(B.graphs[(int)prec] = std::move(L));
}

// Lockstep GMRES(m) of all systems for op x = b ([R][n], Morton), x = 0 on
// entry.  `on` marks the systems to solve (others keep x = 0); tol per
// system relative to ||b_s||.  Returns the Arnoldi steps taken.  TV: the
// type of the Krylov vectors and of their CGS2 arithmetic (FP64; FP32 for the
// inner solves on the low-precision copies, whose tolerance is far above
// FP32's rounding); Hessenberg, rotations, x and the true residual stay FP64.
template <class TV>
static int gmres_batch_t(Batch &B, hm_dtype prec, const double *b, double *x, const std::vector<int> &on, double tol,
                         int maxit, int &cycles, cudaStream_t s, bool use_graph) {
    const int S = B.S, m = B.m;
    const int64_t vs = B.vstride;
    TV *V = B.basis<TV>(s);
    HM_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * vs, s));
    std::vector<double> bn2 = B.norms2(b, s);
    std::vector<int> act(S);
    std::vector<double> bnorm(S);
    for (int k = 0; k < S; ++k) {
        bnorm[k] = std::sqrt(bn2[k]);
        act[k] = on[k] && bnorm[k] > 0.0;
    }
    if (sizeof(TV) == 8) {
        HM_CUDA_CHECK(cudaMemcpyAsync(V, b, sizeof(double) * vs, cudaMemcpyDeviceToDevice, s));
    } else {
        round_vec_kernel<<<gx(vs), 256, 0, s>>>(b, vs, reinterpret_cast<float *>(V));
        HM_LAUNCH_CHECK();
    }
    int iters = 0;
    bool first = true;
    for (;;) {
        // residual norms of V_0 (b in the first cycle)
        std::vector<double> r2 = first ? bn2 : B.norms2(V, s);
        first = false;
        bool any = false;
        for (int k = 0; k < S; ++k) {
            if (act[k] && std::sqrt(r2[k]) <= tol * bnorm[k]) act[k] = 0;
            any = any || act[k];
        }
        if (!any || iters >= maxit) break;
        ++cycles;
        std::vector<int> cyc = act;
        HM_CUDA_CHECK(cudaMemcpyAsync(B.act.p, act.data(), sizeof(int) * S, cudaMemcpyHostToDevice, s));
        HM_CUDA_CHECK(cudaMemcpyAsync(B.cyc.p, cyc.data(), sizeof(int) * S, cudaMemcpyHostToDevice, s));
        HM_CUDA_CHECK(cudaMemsetAsync(B.kk.p, 0, sizeof(int) * S, s));
        // nrm = ||V_0||^2 per system (already in r2): set g, normalise V_0
        HM_CUDA_CHECK(cudaMemcpyAsync(B.nrm.p, r2.data(), sizeof(double) * S, cudaMemcpyHostToDevice, s));
        bset_g0_kernel<<<(S + 127) / 128, 128, 0, s>>>(S, m, B.cyc.as<int>(), B.nrm.as<double>(), B.g.as<double>());
        HM_LAUNCH_CHECK();
        bscale_kernel<TV><<<B.nitems(), 256, 0, s>>>(B.items.as<Item>(), V, B.n, B.nrm.as<double>(), 1,
                                                     B.cyc.as<int>(), V, nullptr, 0, 0);
        HM_LAUNCH_CHECK();
        std::vector<int> kk(S, 0);
        if (use_graph) {
            const LoopGraph &L = batch_step_graph<TV>(B, prec, s);
            std::vector<double> th(S);
            for (int k = 0; k < S; ++k) th[k] = tol * bnorm[k];
            HM_CUDA_CHECK(cudaMemcpyAsync(B.thr.p, th.data(), sizeof(double) * S, cudaMemcpyHostToDevice, s));
            const LoopCtl hc{0, std::min(m, maxit - iters), 0.0};
            HM_CUDA_CHECK(cudaMemcpyAsync(B.ctl.p, &hc, sizeof(hc), cudaMemcpyHostToDevice, s));
            L.launch(s);
            const int steps = read_scalar(&B.ctl.as<LoopCtl>()->j, s);
            L.count(steps);
            iters += steps;
        }
        for (int j = 0; j < (use_graph ? 0 : m); ++j) {
            TV *vj = V + (int64_t)j * vs;
            TV *w = B.wvec<TV>();
            if (B.precond) {
                TV *z = B.zvec<TV>();
                B.bj(vj, z, prec != HM_F64, s);
                B.apply(prec, z, w, s);
            } else {
                B.apply(prec, vj, w, s);
            }
            // CGS2 per system: h = V^T w, w -= V h, h2 = V^T w, w -= V h2, h += h2
            B.dots(V, j + 1, w, B.cyc.as<int>(), B.h.as<double>(), m + 1, 0, s);
            {
                Trace trace("batch_update", s);
                bsub_kernel<TV><<<B.nitems(), 256, 0, s>>>(B.items.as<Item>(), V, vs, B.n, j + 1, B.h.as<double>(),
                                                           m + 1, B.cyc.as<int>(), w, nullptr);
                HM_LAUNCH_CHECK();
            }
            B.dots(V, j + 1, w, B.cyc.as<int>(), B.h2.as<double>(), m + 1, 0, s);
            {
                Trace trace("batch_update", s);
                bsub_kernel<TV><<<B.nitems(), 256, 0, s>>>(B.items.as<Item>(), V, vs, B.n, j + 1, B.h2.as<double>(),
                                                           m + 1, B.cyc.as<int>(), w, nullptr);
                HM_LAUNCH_CHECK();
            }
            badd_coef_kernel<<<gx((int64_t)S * (j + 1)), 256, 0, s>>>(S, j + 1, m + 1, B.h2.as<double>(),
                                                                     B.h.as<double>(), nullptr);
            HM_LAUNCH_CHECK();
            B.dots(w, 1, w, B.cyc.as<int>(), B.nrm.as<double>(), 1, 0, s);
            bgivens_kernel<<<(S + 127) / 128, 128, 0, s>>>(S, m, j, B.cyc.as<int>(), B.h.as<double>(), m + 1,
                                                          B.nrm.as<double>(), B.H.as<double>(), B.cs.as<double>(),
                                                          B.sn.as<double>(), B.g.as<double>(), B.est.as<double>(),
                                                          B.hn.as<double>(), nullptr, nullptr, nullptr);
            HM_LAUNCH_CHECK();
            std::vector<double> est(S), hn(S);
            HM_CUDA_CHECK(cudaMemcpyAsync(est.data(), B.est.p, sizeof(double) * S, cudaMemcpyDeviceToHost, s));
            HM_CUDA_CHECK(cudaMemcpyAsync(hn.data(), B.hn.p, sizeof(double) * S, cudaMemcpyDeviceToHost, s));
            HM_CUDA_CHECK(cudaStreamSynchronize(s));
            ++iters;
            bool more = false;
            for (int k = 0; k < S; ++k) {
                if (!cyc[k]) continue;
                kk[k] = j + 1;
                if (est[k] <= tol * bnorm[k] || hn[k] == 0.0 || iters >= maxit) cyc[k] = 0;
                more = more || cyc[k];
            }
            if (!more) break;
            HM_CUDA_CHECK(cudaMemcpyAsync(B.cyc.p, cyc.data(), sizeof(int) * S, cudaMemcpyHostToDevice, s));
            bscale_kernel<TV><<<B.nitems(), 256, 0, s>>>(B.items.as<Item>(), w, B.n, B.nrm.as<double>(), 1,
                                                         B.cyc.as<int>(), V + (int64_t)(j + 1) * vs, nullptr, 0, 0);
            HM_LAUNCH_CHECK();
        }
        // x += M^{-1} V y per system (the graph form left k_s on the device)
        if (!use_graph) HM_CUDA_CHECK(cudaMemcpyAsync(B.kk.p, kk.data(), sizeof(int) * S, cudaMemcpyHostToDevice, s));
        btrisolve_kernel<<<(S + 127) / 128, 128, 0, s>>>(S, m, B.kk.as<int>(), B.H.as<double>(), B.g.as<double>(),
                                                        B.y.as<double>());
        HM_LAUNCH_CHECK();
        if (B.precond) {
            HM_CUDA_CHECK(cudaMemsetAsync(B.W.p, 0, sizeof(double) * vs, s));
            badd_kernel<TV><<<B.nitems(), 256, 0, s>>>(B.items.as<Item>(), V, vs, B.n, B.kk.as<int>(),
                                                       B.y.as<double>(), m, B.W.as<double>());
            HM_LAUNCH_CHECK();
            B.bj(B.W.as<double>(), B.Z.as<double>(), prec != HM_F64, s);
            badd_vec_kernel<<<gx(vs), 256, 0, s>>>(B.Z.as<double>(), vs, x);
            HM_LAUNCH_CHECK();
        } else {
            badd_kernel<TV><<<B.nitems(), 256, 0, s>>>(B.items.as<Item>(), V, vs, B.n, B.kk.as<int>(),
                                                       B.y.as<double>(), m, x);
            HM_LAUNCH_CHECK();
        }
        // true residual -> V_0 (systems outside `act` keep their x; their rows of V_0 are not used)
        B.apply(prec, x, B.AX.as<double>(), s);
        bsub_vec_kernel<TV><<<gx(vs), 256, 0, s>>>(b, B.AX.as<double>(), vs, V);
        HM_LAUNCH_CHECK();
    }
    return iters;
}

static int gmres_batch(Batch &B, hm_dtype prec, const double *b, double *x, const std::vector<int> &on, double tol,
                       int maxit, int &cycles, cudaStream_t s, bool use_graph) {
    if (prec != HM_F64 && B.v32)
        return gmres_batch_t<float>(B, prec, b, x, on, tol, maxit, cycles, s, use_graph);
    return gmres_batch_t<double>(B, prec, b, x, on, tol, maxit, cycles, s, use_graph);
}

hm_status solve_batched(const hm_matrix *A, int nrhs, const double *b_orig, double *x_orig, const hm_solve_params &p,
                        cudaStream_t s, hm_solve_info *info) {
    const auto t0 = std::chrono::steady_clock::now();
    const hm_tree *tr = A->tree;
    const int64_t n = tr->n;
    const int64_t vs = (int64_t)nrhs * n;
    DBuf b, x;
    b.alloc(sizeof(double) * vs);
    x.alloc(sizeof(double) * vs);
    for (int r = 0; r < nrhs; ++r) permute_to_morton(tr, b_orig + (int64_t)r * n, b.as<double>() + (int64_t)r * n, s);
    HM_CUDA_CHECK(cudaMemsetAsync(x.p, 0, sizeof(double) * vs, s));
    const bool pc = p.precond == 1;
    if (pc) bj_setup(A, s);
    Batch B(A, nrhs, p.restart, pc, p.refine ? p.inner_dtype : HM_F64, s);
    const int S = B.S;
    int iters = 0, cycles = 0, steps = 0;
    hm_dtype inner_dt = p.refine ? p.inner_dtype : HM_F64;
    std::vector<double> bn2 = B.norms2(b.as<double>(), s);
    std::vector<int> on(S, 1);
    double worst = 0.0;
    hm_status st = HM_OK;
    if (!p.refine) {
        iters = gmres_batch(B, HM_F64, b.as<double>(), x.as<double>(), on, p.rel_tol, p.max_iter, cycles, s,
                            p.use_graph != 0);
        B.apply(HM_F64, x.as<double>(), B.AX.as<double>(), s);
        bsub_vec_kernel<double><<<gx(vs), 256, 0, s>>>(b.as<double>(), B.AX.as<double>(), vs, B.W.as<double>());
        HM_LAUNCH_CHECK();
        std::vector<double> r2 = B.norms2(B.W.as<double>(), s);
        for (int k = 0; k < S; ++k) {
            const double rr = bn2[k] > 0.0 ? std::sqrt(r2[k] / bn2[k]) : 0.0;
            worst = std::max(worst, rr);
        }
        if (worst > p.rel_tol) st = HM_ENOCONV;
    } else {
        if (p.resid_df) B.enable_df();
        DBuf r, d;
        r.alloc(sizeof(double) * vs);
        d.alloc(sizeof(double) * vs);
        HM_CUDA_CHECK(cudaMemcpyAsync(r.p, b.p, sizeof(double) * vs, cudaMemcpyDeviceToDevice, s));
        st = HM_ENOCONV;
        const double stall = p.stall_ratio > 0.0 ? p.stall_ratio : 0.5;
        double prev = 1.0;
        for (;;) {
            std::vector<double> r2 = B.norms2(r.as<double>(), s);
            worst = 0.0;
            for (int k = 0; k < S; ++k) {
                const double rr = bn2[k] > 0.0 ? std::sqrt(r2[k] / bn2[k]) : 0.0;
                on[k] = rr > p.rel_tol;
                worst = std::max(worst, rr);
            }
            if (worst <= p.rel_tol) {
                st = HM_OK;
                break;
            }
            // an outer step that did not contract raises the inner precision
            if (steps > 0 && !(worst <= stall * prev) && inner_dt != HM_F64) {
                inner_dt = raise_inner(A, inner_dt, s);
                if (inner_dt != HM_F64) mrhs_prepare(A, inner_dt, s);
            }
            prev = worst;
            if (steps >= p.max_refine || iters >= p.max_iter) break;
            ++steps;
            iters += gmres_batch(B, inner_dt, r.as<double>(), d.as<double>(), on, p.inner_tol,
                                 p.max_iter - iters, cycles, s, p.use_graph != 0);
            badd_vec_kernel<<<gx(vs), 256, 0, s>>>(d.as<double>(), vs, x.as<double>());
            HM_LAUNCH_CHECK();
            B.apply_outer(x.as<double>(), B.AX.as<double>(), s);
            bsub_vec_kernel<double><<<gx(vs), 256, 0, s>>>(b.as<double>(), B.AX.as<double>(), vs, r.as<double>());
            HM_LAUNCH_CHECK();
        }
    }
    for (int r = 0; r < nrhs; ++r)
        permute_from_morton(tr, x.as<double>() + (int64_t)r * n, 1.0, 0.0, x_orig + (int64_t)r * n, s);
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
    if (mrhs_error(A, s)) fail(HM_ETIMEOUT, "a bounded wait of the tensor-memory row pass gave up");
    if (info) {
        info->status = st;
        info->iters = iters;
        info->restarts = cycles;
        info->refine_steps = steps;
        info->rel_resid = worst;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->inner_dtype = (int32_t)inner_dt;
        info->kappa_est = 0.0;  // not estimated by the lockstep solver
    }
    return st;
}

}  // namespace hm
