// tree.cu -- panels, Morton order, cluster tree and block cluster tree.
//
// Sec. 3.1 ("Spatial data structure", "Block cluster tree traversal") and
// Sec. 2.3 (conditions (C1)-(C4), Algorithm 1, admissibility Eq. 5).  All
// integer results are bit-exact: every floating-point step that decides an
// integer (centroid, quantisation, box extents, admissibility) is written
// with explicitly rounded operations (__dadd_rn etc.), so no FMA contraction
// can change a decision.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <numeric>

#include "ff.cuh"

namespace hm {

// ----------------------------------------------------------------------------
// kernels
// ----------------------------------------------------------------------------
__global__ void check_tris_kernel(const int32_t *T, int64_t n, int64_t nv, int *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x)
        if (T[i] < 0 || T[i] >= nv) atomicExch(bad, 1);
}

// centroid c_i = ((v0 + v1) + v2) / 3, original order
__global__ void centroid_kernel(const double *V, const int32_t *T, int64_t n, double *cent) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double *a = V + 3 * (int64_t)T[3 * i], *b = V + 3 * (int64_t)T[3 * i + 1],
                     *c = V + 3 * (int64_t)T[3 * i + 2];
        for (int d = 0; d < 3; ++d) cent[3 * i + d] = __ddiv_rn(__dadd_rn(__dadd_rn(a[d], b[d]), c[d]), 3.0);
    }
}

// per-block min / max of the centroids -> part[block][6]
__global__ void bbox_partial_kernel(const double *cent, int64_t n, double *part) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], cent[3 * i + d]);
            hi[d] = fmax(hi[d], cent[3 * i + d]);
        }
    __shared__ double s[6][32];
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int d = 0; d < 3; ++d) { s[d][warp] = lo[d]; s[3 + d][warp] = hi[d]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
            for (int d = 0; d < 3; ++d) {
                s[d][0] = fmin(s[d][0], s[d][w]);
                s[3 + d][0] = fmax(s[3 + d][0], s[3 + d][w]);
            }
        for (int k = 0; k < 6; ++k) part[6 * blockIdx.x + k] = s[k][0];
    }
}

// lo, and the grid scale s = 2^21 / ext with ext = max_a (hi_a - lo_a) -> out[4]
__global__ void bbox_final_kernel(const double *part, int nb, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], part[6 * b + d]);
            hi[d] = fmax(hi[d], part[6 * b + 3 + d]);
        }
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) ext = fmax(ext, __dsub_rn(hi[d], lo[d]));
    out[0] = lo[0];
    out[1] = lo[1];
    out[2] = lo[2];
    out[3] = ext > 0.0 ? __ddiv_rn(2097152.0, ext) : 0.0;
}

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    // bit b of v -> bit 3b (21 bits)
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x001f00000000ffffull;
    v = (v | (v << 16)) & 0x001f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// q_a = min(2^21 - 1, floor((c_a - lo_a) * s)); code = x bits at 3b+2, y at 3b+1, z at 3b.
// grid[4 g ..]: the cube of geometry g (gid[i] = geometry of panel i; NULL = one geometry)
__global__ void morton_kernel(const double *cent, int64_t n, const double *grid, const int32_t *gid, uint64_t *code,
                              int32_t *idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double *gr = grid + 4 * (gid ? gid[i] : 0);
        const double s = gr[3];
        uint64_t q[3];
        const double lo[3] = {gr[0], gr[1], gr[2]};
        for (int d = 0; d < 3; ++d) {
            double t = floor(__dmul_rn(__dsub_rn(cent[3 * i + d], lo[d]), s));
            uint64_t v = (uint64_t)t;
            q[d] = v > 2097151ull ? 2097151ull : v;
        }
        code[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
        idx[i] = (int32_t)i;
    }
}

// gid[i] = g for the panels [off[g], off[g + 1]) of the input order
__global__ void geom_id_kernel(const int64_t *off, int G, int64_t n, int32_t *gid) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = G;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= i) lo = mid;
            else hi = mid;
        }
        gid[i] = lo;
    }
}

// key[m] = gid[perm[m]] (second, stable pass of the (geometry, code) sort)
__global__ void gather_gid_kernel(const int32_t *gid, const int32_t *perm, int64_t n, uint64_t *key) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x)
        key[m] = (uint64_t)gid[perm[m]];
}

// panel table in Morton order
__global__ void panel_table_kernel(const double *V, const int32_t *T, const int32_t *perm, const double *cent,
                                   int64_t n, int64_t npad, QuadParams qp, double *pt, float *pf, double *cent_s,
                                   int32_t *trim, int32_t *iperm) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = perm[k];
        const int32_t t0 = T[3 * (int64_t)i], t1 = T[3 * (int64_t)i + 1], t2 = T[3 * (int64_t)i + 2];
        const double *a = V + 3 * (int64_t)t0, *b = V + 3 * (int64_t)t1, *c = V + 3 * (int64_t)t2;
        // float-pair record: the centroid as (h, l) and every quadrature point
        // as an offset from that represented centroid h + l (exact in FP64),
        // so a point's representation error is relative to the panel size
        double cr[3];
        for (int d = 0; d < 3; ++d) {
            float h, l;
            split_double(cent[3 * (int64_t)i + d], h, l);
            pf[(int64_t)(PF_CH + d) * npad + k] = h;
            pf[(int64_t)(PF_CL + d) * npad + k] = l;
            cr[d] = __dadd_rn((double)h, (double)l);
        }
        for (int q = 0; q < NQ; ++q)
            for (int d = 0; d < 3; ++d) {
                const double xq = __dadd_rn(__dadd_rn(__dmul_rn(qp.bary[q][0], a[d]), __dmul_rn(qp.bary[q][1], b[d])),
                                            __dmul_rn(qp.bary[q][2], c[d]));
                pt[(int64_t)(7 * d + q) * npad + k] = xq;
                float h, l;
                split_double(__dsub_rn(xq, cr[d]), h, l);
                pf[(int64_t)(PF_AH + 7 * d + q) * npad + k] = h;
                pf[(int64_t)(PF_AL + 7 * d + q) * npad + k] = l;
            }
        pf[(int64_t)(PF_VID + 0) * npad + k] = __int_as_float(t0);
        pf[(int64_t)(PF_VID + 1) * npad + k] = __int_as_float(t1);
        pf[(int64_t)(PF_VID + 2) * npad + k] = __int_as_float(t2);
        double e1[3], e2[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = __dsub_rn(b[d], a[d]);
            e2[d] = __dsub_rn(c[d], a[d]);
        }
        double x0 = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
        double x1 = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
        double x2 = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
        double nn = __dadd_rn(__dadd_rn(__dmul_rn(x0, x0), __dmul_rn(x1, x1)), __dmul_rn(x2, x2));
        const double area = __dmul_rn(0.5, __dsqrt_rn(nn));
        pt[(int64_t)PT_AREA * npad + k] = area;
        {
            float h, l;
            split_double(area / SQRT_4PI, h, l);
            pf[(int64_t)PF_WA * npad + k] = h;
            pf[(int64_t)(PF_WA + 1) * npad + k] = l;
        }
        pt[(int64_t)(PT_VID + 0) * npad + k] = (double)t0;
        pt[(int64_t)(PT_VID + 1) * npad + k] = (double)t1;
        pt[(int64_t)(PT_VID + 2) * npad + k] = (double)t2;
        for (int d = 0; d < 3; ++d) cent_s[3 * k + d] = cent[3 * (int64_t)i + d];
        trim[3 * k] = t0;
        trim[3 * k + 1] = t1;
        trim[3 * k + 2] = t2;
        iperm[i] = (int32_t)k;
    }
}

// boxes of leaf clusters: one warp per cluster, exact min / max
__global__ void leaf_box_kernel(const double *cent_s, const int32_t *range, const int32_t *child, int64_t nc,
                                double *box) {
    const int lane = threadIdx.x & 31;
    int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (c >= nc || child[c] >= 0) return;
    const int32_t b = range[2 * c], e = range[2 * c + 1];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t k = b + lane; k < e; k += 32)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], cent_s[3 * (int64_t)k + d]);
            hi[d] = fmax(hi[d], cent_s[3 * (int64_t)k + d]);
        }
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    if (lane == 0)
        for (int d = 0; d < 3; ++d) { box[6 * c + d] = lo[d]; box[6 * c + 3 + d] = hi[d]; }
}

// boxes of the non-leaf clusters of one level: union of the two children
__global__ void parent_box_kernel(const int32_t *child, int64_t c0, int64_t c1, double *box) {
    int64_t c = c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= c1 || child[c] < 0) return;
    const int64_t a = child[c], b = a + 1;
    for (int d = 0; d < 3; ++d) {
        box[6 * c + d] = fmin(box[6 * a + d], box[6 * b + d]);
        box[6 * c + 3 + d] = fmax(box[6 * a + 3 + d], box[6 * b + 3 + d]);
    }
}

// Eq. 5 in squared form: min(diam^2) <= eta^2 * dist^2, sums in x, y, z order
__device__ __forceinline__ bool admissible_dev(const double *bt, const double *bs, double eta2) {
    double dt2 = 0.0, ds2 = 0.0, g2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double dt = __dsub_rn(bt[3 + d], bt[d]);
        double ds = __dsub_rn(bs[3 + d], bs[d]);
        double g1 = __dsub_rn(bs[d], bt[3 + d]);
        double gg = __dsub_rn(bt[d], bs[3 + d]);
        double g = 0.0;
        if (g1 > g) g = g1;
        if (gg > g) g = gg;
        if (d == 0) {
            dt2 = __dmul_rn(dt, dt);
            ds2 = __dmul_rn(ds, ds);
            g2 = __dmul_rn(g, g);
        } else {
            dt2 = __dadd_rn(dt2, __dmul_rn(dt, dt));
            ds2 = __dadd_rn(ds2, __dmul_rn(ds, ds));
            g2 = __dadd_rn(g2, __dmul_rn(g, g));
        }
    }
    double mind = dt2 < ds2 ? dt2 : ds2;
    return mind <= __dmul_rn(eta2, g2);
}

// Algorithm 1, one level: 0 = admissible leaf, 1 = dense leaf, 2 = four children.
// counts: adm (1), dense (1, or 2 when the row cluster is split for storage),
// children (4).
__global__ void bt_classify_kernel(const int32_t *cand, int64_t ncand, const int32_t *range, const double *box,
                                   const int32_t *child, int32_t leaf, double eta2, int8_t *flag, int64_t *c_adm,
                                   int64_t *c_den, int64_t *c_sub) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncand;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = cand[2 * i], s = cand[2 * i + 1];
        const int32_t szt = range[2 * t + 1] - range[2 * t], szs = range[2 * s + 1] - range[2 * s];
        const bool adm = admissible_dev(box + 6 * (int64_t)t, box + 6 * (int64_t)s, eta2);
        int8_t f;
        if (!adm && szt > leaf && szs > leaf) f = 2;
        else if (adm) f = 0;
        else f = 1;
        flag[i] = f;
        c_adm[i] = f == 0;
        c_den[i] = f == 1 ? (szt > leaf ? 2 : 1) : 0;
        c_sub[i] = f == 2 ? 4 : 0;
    }
}

__global__ void bt_emit_kernel(const int32_t *cand, int64_t ncand, const int32_t *range, const int32_t *child,
                               const int8_t *flag, const int64_t *o_adm, const int64_t *o_den, const int64_t *o_sub,
                               int32_t *adm_out, int32_t *den_out, int32_t *next) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncand;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = cand[2 * i], s = cand[2 * i + 1];
        const int8_t f = flag[i];
        if (f == 0) {
            int32_t *o = adm_out + 4 * o_adm[i];
            o[0] = range[2 * t]; o[1] = range[2 * t + 1]; o[2] = range[2 * s]; o[3] = range[2 * s + 1];
        } else if (f == 1) {
            int32_t *o = den_out + 4 * o_den[i];
            if (child[t] >= 0) {
                // non-leaf row cluster next to a leaf column cluster: stored as
                // its two children's rows (same entries, leaf-cluster row panels)
                const int32_t a = child[t], b = a + 1;
                o[0] = range[2 * a]; o[1] = range[2 * a + 1]; o[2] = range[2 * s]; o[3] = range[2 * s + 1];
                o[4] = range[2 * b]; o[5] = range[2 * b + 1]; o[6] = range[2 * s]; o[7] = range[2 * s + 1];
            } else {
                o[0] = range[2 * t]; o[1] = range[2 * t + 1]; o[2] = range[2 * s]; o[3] = range[2 * s + 1];
            }
        } else {
            int32_t *o = next + 2 * o_sub[i];
            const int32_t ta = child[t], sa = child[s];
            o[0] = ta;     o[1] = sa;
            o[2] = ta;     o[3] = sa + 1;
            o[4] = ta + 1; o[5] = sa;
            o[6] = ta + 1; o[7] = sa + 1;
        }
    }
}

__global__ void dense_keys_kernel(const int32_t *den, int64_t nd, uint64_t *key, int32_t *idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd; i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = ((uint64_t)(uint32_t)den[4 * i] << 32) | (uint32_t)den[4 * i + 2];
        idx[i] = (int32_t)i;
    }
}

__global__ void gather_rows4_kernel(const int32_t *src, const int32_t *idx, int64_t n, int32_t *dst, int64_t *width) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *s = src + 4 * (int64_t)idx[i];
        for (int k = 0; k < 4; ++k) dst[4 * i + k] = s[k];
        width[i] = s[3] - s[2];
    }
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t n, int32_t v, int stride) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid * stride] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// per leaf row cluster: first dense block, padded panel width, panel size
__global__ void rho_kernel(const int32_t *den_sorted, int64_t nd, const int64_t *wpre, const int32_t *leaf_begin,
                           int64_t nleaf, int64_t *rho_first, int32_t *rho_K, int64_t *rho_size,
                           int64_t *rho_kpad) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nleaf; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = lower_bound_i32(den_sorted, nd, leaf_begin[r], 4);
        const int64_t e = lower_bound_i32(den_sorted, nd, leaf_begin[r + 1], 4);
        const int64_t K = wpre[e] - wpre[s];
        const int64_t Kp = (K + 7) / 8 * 8;
        rho_first[r] = s;
        rho_K[r] = (int32_t)Kp;
        rho_size[r] = (int64_t)(leaf_begin[r + 1] - leaf_begin[r]) * Kp;
        rho_kpad[r] = Kp;
    }
}

// dense block -> arena base / ld, and the panel's column index list
// (padding columns keep index 0 and value 0)
__global__ void dense_layout_kernel(const int32_t *den_sorted, int64_t nd, const int64_t *wpre,
                                    const int32_t *leaf_begin, int64_t nleaf, const int64_t *rho_first,
                                    const int64_t *rho_off, const int64_t *rho_colptr, const int32_t *rho_K,
                                    int64_t *base, int32_t *ld, int32_t *colidx) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nd; b += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rb = den_sorted[4 * b], cb = den_sorted[4 * b + 2], ce = den_sorted[4 * b + 3];
        const int64_t r = lower_bound_i32(leaf_begin, nleaf, rb, 1);
        const int64_t koff = wpre[b] - wpre[rho_first[r]];
        base[b] = rho_off[r] + koff;
        ld[b] = rho_K[r];
        for (int32_t j = 0; j < ce - cb; ++j) colidx[rho_colptr[r] + koff + j] = cb + j;
    }
}

// admissible block -> number of leaf clusters its rows (side = 0) or its
// columns (side = 2) cover
__global__ void lr_count_kernel(const int32_t *adm, int64_t na, const int32_t *leaf_begin, int64_t nleaf, int side,
                                int64_t *cnt) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l0 = lower_bound_i32(leaf_begin, nleaf + 1, adm[4 * b + side], 1);
        const int64_t l1 = lower_bound_i32(leaf_begin, nleaf + 1, adm[4 * b + side + 1], 1);
        cnt[b] = l1 - l0;
    }
}

__global__ void lr_pairs_kernel(const int32_t *adm, int64_t na, const int32_t *leaf_begin, int64_t nleaf, int side,
                                const int64_t *off, uint64_t *key, int32_t *val) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < na; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l0 = lower_bound_i32(leaf_begin, nleaf + 1, adm[4 * b + side], 1);
        const int64_t l1 = lower_bound_i32(leaf_begin, nleaf + 1, adm[4 * b + side + 1], 1);
        for (int64_t l = l0; l < l1; ++l) {
            key[off[b] + l - l0] = ((uint64_t)l << 32) | (uint64_t)b;
            val[off[b] + l - l0] = (int32_t)b;
        }
    }
}

__global__ void lr_rowcount_kernel(const uint64_t *key, int64_t np, int64_t *rowcnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long *>(rowcnt + (key[i] >> 32)), 1ull);
}

__global__ void valence_kernel(const int32_t *T, int64_t n, int32_t *val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(val + T[i], 1);
}

__global__ void square_kernel(const int32_t *v, int64_t n, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)v[i] * v[i];
}

// keys (row_begin << 32 | col_begin) of a leaf list, with identity payloads
__global__ void leaf_keys_kernel(const int32_t *q, int64_t n, uint64_t *key, int32_t *idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = ((uint64_t)(uint32_t)q[4 * i] << 32) | (uint32_t)q[4 * i + 2];
        idx[i] = (int32_t)i;
    }
}

// Transposed partner of each leaf: the leaf with exactly the swapped row and
// column ranges (binary search over the sorted keys), or -1.
__global__ void partner_kernel(const int32_t *q, int64_t n, const uint64_t *skey, const int32_t *sidx, int32_t *tp) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t want = ((uint64_t)(uint32_t)q[4 * i + 2] << 32) | (uint32_t)q[4 * i];
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (skey[mid] < want) lo = mid + 1;
            else hi = mid;
        }
        int32_t r = -1;
        if (lo < n && skey[lo] == want) {
            const int32_t j = sidx[lo];
            if (q[4 * j + 1] == q[4 * i + 3] && q[4 * j + 3] == q[4 * i + 1]) r = j;
        }
        tp[i] = r;
    }
}

__global__ void block_size_kernel(const int32_t *quad, int64_t n, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)(quad[4 * i + 1] - quad[4 * i]) * (quad[4 * i + 3] - quad[4 * i + 2]);
}

__global__ void i64_from_i32_diff_kernel(const int32_t *quad, int64_t n, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)(quad[4 * i + 1] - quad[4 * i]) + (quad[4 * i + 3] - quad[4 * i + 2]);
}

// ----------------------------------------------------------------------------
// host orchestration
// ----------------------------------------------------------------------------
static unsigned grid_for(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (unsigned)b;
}

hm_tree *build_tree_impl(const double *d_V, int64_t nv, const int32_t *d_T, int64_t n, const hm_tree_params &prm,
                         const std::vector<int64_t> &goff_in, cudaStream_t s) {
    // geometries: triangle ranges [goff[g], goff[g + 1]) of the input (one geometry by default)
    std::vector<int64_t> goff = goff_in.empty() ? std::vector<int64_t>{0, n} : goff_in;
    const int G = (int)goff.size() - 1;
    auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<hm_tree> tr(new hm_tree());
    tr->n = n;
    tr->nv = nv;
    tr->npad = (n + 7) / 8 * 8;
    tr->leaf = prm.leaf_size;
    tr->eta = prm.eta;
    const int64_t npad = tr->npad;

    // copies of the caller's mesh, index check
    tr->V.alloc(sizeof(double) * 3 * nv);
    HM_CUDA_CHECK(cudaMemcpyAsync(tr->V.p, d_V, sizeof(double) * 3 * nv, cudaMemcpyDeviceToDevice, s));
    DBuf T;
    T.alloc(sizeof(int32_t) * 3 * n);
    HM_CUDA_CHECK(cudaMemcpyAsync(T.p, d_T, sizeof(int32_t) * 3 * n, cudaMemcpyDeviceToDevice, s));
    {
        DBuf bad;
        bad.alloc(sizeof(int));
        HM_CUDA_CHECK(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
        check_tris_kernel<<<grid_for(3 * n), 256, 0, s>>>(T.as<int32_t>(), n, nv, bad.as<int>());
        HM_LAUNCH_CHECK();
        if (read_scalar(bad.as<int>(), s)) fail(HM_EINVAL, "a triangle vertex index is outside [0, n_vertices)");
    }
    const double *V = tr->V.as<double>();

    // a1 / a2: centroids, bounding cube, Morton codes
    DBuf cent;
    cent.alloc(sizeof(double) * 3 * n);
    centroid_kernel<<<grid_for(n), 256, 0, s>>>(V, T.as<int32_t>(), n, cent.as<double>());
    HM_LAUNCH_CHECK();
    // the bounding cube of every geometry
    const int nbb = 256;
    DBuf part, grid;
    part.alloc(sizeof(double) * 6 * nbb);
    grid.alloc(sizeof(double) * 4 * G);
    for (int g = 0; g < G; ++g) {
        const int64_t cnt = goff[g + 1] - goff[g];
        const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(nbb, (cnt + 255) / 256));
        bbox_partial_kernel<<<nb, 256, 0, s>>>(cent.as<double>() + 3 * goff[g], cnt, part.as<double>());
        HM_LAUNCH_CHECK();
        bbox_final_kernel<<<1, 32, 0, s>>>(part.as<double>(), nb, grid.as<double>() + 4 * g);
        HM_LAUNCH_CHECK();
    }
    DBuf gid;
    if (G > 1) {
        DBuf d_goff;
        d_goff.alloc(sizeof(int64_t) * (G + 1));
        HM_CUDA_CHECK(cudaMemcpyAsync(d_goff.p, goff.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, s));
        gid.alloc(sizeof(int32_t) * n);
        geom_id_kernel<<<grid_for(n), 256, 0, s>>>(d_goff.as<int64_t>(), G, n, gid.as<int32_t>());
        HM_LAUNCH_CHECK();
        HM_CUDA_CHECK(cudaStreamSynchronize(s));
    }
    DBuf code, code_tmp, idx_tmp;
    code.alloc(sizeof(uint64_t) * n);
    code_tmp.alloc(sizeof(uint64_t) * n);
    idx_tmp.alloc(sizeof(int32_t) * n);
    tr->perm.alloc(sizeof(int32_t) * n);
    morton_kernel<<<grid_for(n), 256, 0, s>>>(cent.as<double>(), n, grid.as<double>(), G > 1 ? gid.as<int32_t>() : nullptr,
                                             code.as<uint64_t>(), tr->perm.as<int32_t>());
    HM_LAUNCH_CHECK();
    // a3: stable sort by (code, original index), then, for several
    // geometries, stable by geometry: the order is (geometry, code, index)
    radix_sort_u64(code.as<uint64_t>(), tr->perm.as<int32_t>(), code_tmp.as<uint64_t>(), idx_tmp.as<int32_t>(), n, 63,
                   s);
    if (G > 1) {
        int bits = 1;
        while ((1 << bits) < G) ++bits;
        gather_gid_kernel<<<grid_for(n), 256, 0, s>>>(gid.as<int32_t>(), tr->perm.as<int32_t>(), n, code.as<uint64_t>());
        HM_LAUNCH_CHECK();
        radix_sort_u64(code.as<uint64_t>(), tr->perm.as<int32_t>(), code_tmp.as<uint64_t>(), idx_tmp.as<int32_t>(), n,
                       bits, s);
    }
    tr->geom_off = goff;

    // panel table in Morton order
    const QuadParams qp = make_quad(1);
    tr->pt.alloc(sizeof(double) * PT_ROWS * npad);
    HM_CUDA_CHECK(cudaMemsetAsync(tr->pt.p, 0, sizeof(double) * PT_ROWS * npad, s));
    tr->pf.alloc(sizeof(float) * PF_ROWS * npad);
    HM_CUDA_CHECK(cudaMemsetAsync(tr->pf.p, 0, sizeof(float) * PF_ROWS * npad, s));
    tr->cent.alloc(sizeof(double) * 3 * n);
    tr->trim.alloc(sizeof(int32_t) * 3 * n);
    tr->iperm.alloc(sizeof(int32_t) * n);
    panel_table_kernel<<<grid_for(n), 256, 0, s>>>(V, T.as<int32_t>(), tr->perm.as<int32_t>(), cent.as<double>(), n,
                                                  npad, qp, tr->pt.as<double>(), tr->pf.as<float>(),
                                                  tr->cent.as<double>(),
                                                  tr->trim.as<int32_t>(), tr->iperm.as<int32_t>());
    HM_LAUNCH_CHECK();

    // a4: cardinality-based cluster tree (integer only, host), boxes on device
    std::vector<int32_t> range, child;
    std::vector<int64_t> level_start;
    for (int g = 0; g < G; ++g) {  // one root per geometry
        range.push_back((int32_t)goff[g]);
        range.push_back((int32_t)goff[g + 1]);
        child.push_back(-1);
    }
    level_start.push_back(0);
    int64_t lb = 0, le = G;
    int32_t max_leaf = 0;
    std::vector<int32_t> leaf_begin;
    while (lb < le) {
        level_start.push_back(le);
        for (int64_t c = lb; c < le; ++c) {
            const int32_t b = range[2 * c], e = range[2 * c + 1];
            if (e - b > prm.leaf_size) {
                const int32_t m = b + (e - b) / 2;
                child[c] = (int32_t)(range.size() / 2);
                range.push_back(b); range.push_back(m); child.push_back(-1);
                range.push_back(m); range.push_back(e); child.push_back(-1);
            } else {
                leaf_begin.push_back(b);
                max_leaf = std::max(max_leaf, e - b);
            }
        }
        lb = le;
        le = (int64_t)range.size() / 2;
    }
    const int64_t nc = (int64_t)child.size();
    tr->n_clusters = nc;
    tr->depth = (int32_t)level_start.size() - 2;
    std::sort(leaf_begin.begin(), leaf_begin.end());
    tr->n_leaf = (int64_t)leaf_begin.size();
    leaf_begin.push_back((int32_t)n);
    tr->max_leaf = max_leaf;
    tr->cl_range.alloc(sizeof(int32_t) * 2 * nc);
    DBuf d_child;
    d_child.alloc(sizeof(int32_t) * nc);
    tr->cl_box.alloc(sizeof(double) * 6 * nc);
    tr->leaf_begin.alloc(sizeof(int32_t) * leaf_begin.size());
    HM_CUDA_CHECK(cudaMemcpyAsync(tr->cl_range.p, range.data(), sizeof(int32_t) * 2 * nc, cudaMemcpyHostToDevice, s));
    HM_CUDA_CHECK(cudaMemcpyAsync(d_child.p, child.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice, s));
    HM_CUDA_CHECK(cudaMemcpyAsync(tr->leaf_begin.p, leaf_begin.data(), sizeof(int32_t) * leaf_begin.size(),
                                  cudaMemcpyHostToDevice, s));
    leaf_box_kernel<<<grid_for(32 * nc), 256, 0, s>>>(tr->cent.as<double>(), tr->cl_range.as<int32_t>(),
                                                      d_child.as<int32_t>(), nc, tr->cl_box.as<double>());
    HM_LAUNCH_CHECK();
    for (int64_t L = (int64_t)level_start.size() - 2; L >= 0; --L) {
        const int64_t c0 = level_start[L], c1 = level_start[L + 1];
        if (c1 > c0)
            parent_box_kernel<<<grid_for(c1 - c0), 256, 0, s>>>(d_child.as<int32_t>(), c0, c1, tr->cl_box.as<double>());
        HM_LAUNCH_CHECK();
    }

    // a5: block cluster tree, level by level (Algorithm 1 from I x I)
    std::vector<DBuf> adm_parts, den_parts;
    std::vector<int64_t> adm_cnt, den_cnt;
    DBuf cand;
    cand.alloc(sizeof(int32_t) * 2 * G);
    {
        std::vector<int32_t> roots(2 * G);  // (root_g, root_g): blocks never pair two geometries
        for (int g = 0; g < G; ++g) roots[2 * g] = roots[2 * g + 1] = g;
        HM_CUDA_CHECK(cudaMemcpyAsync(cand.p, roots.data(), sizeof(int32_t) * 2 * G, cudaMemcpyHostToDevice, s));
        HM_CUDA_CHECK(cudaStreamSynchronize(s));
    }
    int64_t ncand = G;
    const double eta2 = prm.eta * prm.eta;
    while (ncand > 0) {
        DBuf flag, ca, cd, cs;
        flag.alloc(ncand);
        ca.alloc(sizeof(int64_t) * ncand);
        cd.alloc(sizeof(int64_t) * ncand);
        cs.alloc(sizeof(int64_t) * ncand);
        bt_classify_kernel<<<grid_for(ncand), 256, 0, s>>>(
            cand.as<int32_t>(), ncand, tr->cl_range.as<int32_t>(), tr->cl_box.as<double>(), d_child.as<int32_t>(),
            prm.leaf_size, eta2, flag.as<int8_t>(), ca.as<int64_t>(), cd.as<int64_t>(), cs.as<int64_t>());
        HM_LAUNCH_CHECK();
        const int64_t na = exclusive_scan_i64(ca.as<int64_t>(), ca.as<int64_t>(), ncand, s);
        const int64_t nd = exclusive_scan_i64(cd.as<int64_t>(), cd.as<int64_t>(), ncand, s);
        const int64_t ns = exclusive_scan_i64(cs.as<int64_t>(), cs.as<int64_t>(), ncand, s);
        DBuf ao, dout, next;
        ao.alloc(sizeof(int32_t) * 4 * std::max<int64_t>(na, 1));
        dout.alloc(sizeof(int32_t) * 4 * std::max<int64_t>(nd, 1));
        next.alloc(sizeof(int32_t) * 2 * std::max<int64_t>(ns, 1));
        bt_emit_kernel<<<grid_for(ncand), 256, 0, s>>>(cand.as<int32_t>(), ncand, tr->cl_range.as<int32_t>(),
                                                       d_child.as<int32_t>(), flag.as<int8_t>(), ca.as<int64_t>(),
                                                       cd.as<int64_t>(), cs.as<int64_t>(), ao.as<int32_t>(),
                                                       dout.as<int32_t>(), next.as<int32_t>());
        HM_LAUNCH_CHECK();
        if (na) { adm_parts.push_back(std::move(ao)); adm_cnt.push_back(na); }
        if (nd) { den_parts.push_back(std::move(dout)); den_cnt.push_back(nd); }
        cand = std::move(next);
        ncand = ns;
    }
    const int64_t n_adm = std::accumulate(adm_cnt.begin(), adm_cnt.end(), (int64_t)0);
    const int64_t n_den = std::accumulate(den_cnt.begin(), den_cnt.end(), (int64_t)0);
    tr->n_adm = n_adm;
    tr->n_dense = n_den;
    tr->adm.alloc(sizeof(int32_t) * 4 * std::max<int64_t>(n_adm, 1));
    DBuf den_all;
    den_all.alloc(sizeof(int32_t) * 4 * std::max<int64_t>(n_den, 1));
    {
        int64_t o = 0;
        for (size_t k = 0; k < adm_parts.size(); ++k) {
            HM_CUDA_CHECK(cudaMemcpyAsync(tr->adm.as<int32_t>() + 4 * o, adm_parts[k].p, sizeof(int32_t) * 4 * adm_cnt[k],
                                          cudaMemcpyDeviceToDevice, s));
            o += adm_cnt[k];
        }
        o = 0;
        for (size_t k = 0; k < den_parts.size(); ++k) {
            HM_CUDA_CHECK(cudaMemcpyAsync(den_all.as<int32_t>() + 4 * o, den_parts[k].p, sizeof(int32_t) * 4 * den_cnt[k],
                                          cudaMemcpyDeviceToDevice, s));
            o += den_cnt[k];
        }
    }
    adm_parts.clear();
    den_parts.clear();

    // dense leaves sorted by (row_begin, col_begin), grouped in leaf row panels
    {
        DBuf key, kt, idx, it, width;
        key.alloc(sizeof(uint64_t) * n_den);
        kt.alloc(sizeof(uint64_t) * n_den);
        idx.alloc(sizeof(int32_t) * n_den);
        it.alloc(sizeof(int32_t) * n_den);
        width.alloc(sizeof(int64_t) * (n_den + 1));
        dense_keys_kernel<<<grid_for(n_den), 256, 0, s>>>(den_all.as<int32_t>(), n_den, key.as<uint64_t>(),
                                                          idx.as<int32_t>());
        HM_LAUNCH_CHECK();
        radix_sort_u64(key.as<uint64_t>(), idx.as<int32_t>(), kt.as<uint64_t>(), it.as<int32_t>(), n_den, 64, s);
        tr->dense.alloc(sizeof(int32_t) * 4 * n_den);
        gather_rows4_kernel<<<grid_for(n_den), 256, 0, s>>>(den_all.as<int32_t>(), idx.as<int32_t>(), n_den,
                                                            tr->dense.as<int32_t>(), width.as<int64_t>());
        HM_LAUNCH_CHECK();
        HM_CUDA_CHECK(cudaMemsetAsync(width.as<int64_t>() + n_den, 0, sizeof(int64_t), s));
        exclusive_scan_i64(width.as<int64_t>(), width.as<int64_t>(), n_den + 1, s);
        const int64_t nl = tr->n_leaf;
        DBuf rho_first, rho_size, kpad;
        rho_first.alloc(sizeof(int64_t) * nl);
        rho_size.alloc(sizeof(int64_t) * (nl + 1));
        kpad.alloc(sizeof(int64_t) * (nl + 1));
        tr->rho_K.alloc(sizeof(int32_t) * nl);
        tr->rho_colptr.alloc(sizeof(int64_t) * (nl + 1));
        tr->rho_off.alloc(sizeof(int64_t) * (nl + 1));
        rho_kernel<<<grid_for(nl), 256, 0, s>>>(tr->dense.as<int32_t>(), n_den, width.as<int64_t>(),
                                                tr->leaf_begin.as<int32_t>(), nl, rho_first.as<int64_t>(),
                                                tr->rho_K.as<int32_t>(), rho_size.as<int64_t>(),
                                                kpad.as<int64_t>());
        HM_LAUNCH_CHECK();
        HM_CUDA_CHECK(cudaMemsetAsync(rho_size.as<int64_t>() + nl, 0, sizeof(int64_t), s));
        HM_CUDA_CHECK(cudaMemsetAsync(kpad.as<int64_t>() + nl, 0, sizeof(int64_t), s));
        const int64_t total_kp = exclusive_scan_i64(kpad.as<int64_t>(), tr->rho_colptr.as<int64_t>(), nl + 1, s);
        tr->dense_entries = exclusive_scan_i64(rho_size.as<int64_t>(), tr->rho_off.as<int64_t>(), nl + 1, s);
        tr->dense_base.alloc(sizeof(int64_t) * n_den);
        tr->dense_ld.alloc(sizeof(int32_t) * n_den);
        tr->colidx.alloc(sizeof(int32_t) * std::max<int64_t>(total_kp, 1));
        HM_CUDA_CHECK(cudaMemsetAsync(tr->colidx.p, 0, sizeof(int32_t) * std::max<int64_t>(total_kp, 1), s));
        dense_layout_kernel<<<grid_for(n_den), 256, 0, s>>>(
            tr->dense.as<int32_t>(), n_den, width.as<int64_t>(), tr->leaf_begin.as<int32_t>(), nl,
            rho_first.as<int64_t>(), tr->rho_off.as<int64_t>(), tr->rho_colptr.as<int64_t>(),
            tr->rho_K.as<int32_t>(), tr->dense_base.as<int64_t>(), tr->dense_ld.as<int32_t>(),
            tr->colidx.as<int32_t>());
        HM_LAUNCH_CHECK();
        // stored entries without padding: sum over dense leaves of m * n
        DBuf mn;
        mn.alloc(sizeof(int64_t) * (n_den + 1));
        block_size_kernel<<<grid_for(n_den), 256, 0, s>>>(tr->dense.as<int32_t>(), n_den, mn.as<int64_t>());
        HM_LAUNCH_CHECK();
        tr->dense_true = exclusive_scan_i64(mn.as<int64_t>(), mn.as<int64_t>(), n_den, s);
        // transposed partners (the list is sorted by (row_begin, col_begin))
        tr->dense_tp.alloc(sizeof(int32_t) * std::max<int64_t>(n_den, 1));
        if (n_den) {
            DBuf k2, i2;
            k2.alloc(sizeof(uint64_t) * n_den);
            i2.alloc(sizeof(int32_t) * n_den);
            leaf_keys_kernel<<<grid_for(n_den), 256, 0, s>>>(tr->dense.as<int32_t>(), n_den, k2.as<uint64_t>(),
                                                             i2.as<int32_t>());
            HM_LAUNCH_CHECK();
            partner_kernel<<<grid_for(n_den), 256, 0, s>>>(tr->dense.as<int32_t>(), n_den, k2.as<uint64_t>(),
                                                           i2.as<int32_t>(), tr->dense_tp.as<int32_t>());
            HM_LAUNCH_CHECK();
        }
    }
    // largest dense dimension (for the TMA box)
    tr->max_dense_dim = std::max(max_leaf, std::min<int32_t>((int32_t)n, max_leaf + 1));

    // admissible leaves: sum of |tau| + |sigma|, and for every leaf cluster the
    // admissible leaves whose rows (resp. columns) cover it, ascending
    {
        const int64_t nl = tr->n_leaf;
        if (n_adm) {
            DBuf cnt;
            cnt.alloc(sizeof(int64_t) * (n_adm + 1));
            i64_from_i32_diff_kernel<<<grid_for(n_adm), 256, 0, s>>>(tr->adm.as<int32_t>(), n_adm, cnt.as<int64_t>());
            HM_LAUNCH_CHECK();
            tr->adm_rows_cols = exclusive_scan_i64(cnt.as<int64_t>(), cnt.as<int64_t>(), n_adm, s);
        }
        auto build_csr = [&](int side, DBuf &ptr, DBuf &list, DBuf *bptr) {
            ptr.alloc(sizeof(int64_t) * (nl + 1));
            HM_CUDA_CHECK(cudaMemsetAsync(ptr.p, 0, sizeof(int64_t) * (nl + 1), s));
            DBuf cnt;
            cnt.alloc(sizeof(int64_t) * (n_adm + 1));
            HM_CUDA_CHECK(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * (n_adm + 1), s));
            if (n_adm) {
                lr_count_kernel<<<grid_for(n_adm), 256, 0, s>>>(tr->adm.as<int32_t>(), n_adm,
                                                                tr->leaf_begin.as<int32_t>(), nl, side,
                                                                cnt.as<int64_t>());
                HM_LAUNCH_CHECK();
            }
            const int64_t np = exclusive_scan_i64(cnt.as<int64_t>(), cnt.as<int64_t>(), n_adm + 1, s);
            list.alloc(sizeof(int32_t) * std::max<int64_t>(np, 1));
            if (np) {
                DBuf key, kt, vt;
                key.alloc(sizeof(uint64_t) * np);
                kt.alloc(sizeof(uint64_t) * np);
                vt.alloc(sizeof(int32_t) * np);
                lr_pairs_kernel<<<grid_for(n_adm), 256, 0, s>>>(tr->adm.as<int32_t>(), n_adm,
                                                                tr->leaf_begin.as<int32_t>(), nl, side,
                                                                cnt.as<int64_t>(), key.as<uint64_t>(),
                                                                list.as<int32_t>());
                HM_LAUNCH_CHECK();
                radix_sort_u64(key.as<uint64_t>(), list.as<int32_t>(), kt.as<uint64_t>(), vt.as<int32_t>(), np, 64,
                               s);
                lr_rowcount_kernel<<<grid_for(np), 256, 0, s>>>(key.as<uint64_t>(), np, ptr.as<int64_t>());
                HM_LAUNCH_CHECK();
                exclusive_scan_i64(ptr.as<int64_t>(), ptr.as<int64_t>(), nl + 1, s);
            }
            if (bptr) *bptr = std::move(cnt);
        };
        build_csr(0, tr->lr_rowptr, tr->lr_list, &tr->lr_browptr);
        build_csr(2, tr->lr_colptr, tr->lr_collist, &tr->lr_bcolptr);
        // transposed partners of the admissible leaves
        tr->adm_tp.alloc(sizeof(int32_t) * std::max<int64_t>(n_adm, 1));
        if (n_adm) {
            DBuf k2, i2, kt, it;
            k2.alloc(sizeof(uint64_t) * n_adm);
            i2.alloc(sizeof(int32_t) * n_adm);
            kt.alloc(sizeof(uint64_t) * n_adm);
            it.alloc(sizeof(int32_t) * n_adm);
            leaf_keys_kernel<<<grid_for(n_adm), 256, 0, s>>>(tr->adm.as<int32_t>(), n_adm, k2.as<uint64_t>(),
                                                             i2.as<int32_t>());
            HM_LAUNCH_CHECK();
            radix_sort_u64(k2.as<uint64_t>(), i2.as<int32_t>(), kt.as<uint64_t>(), it.as<int32_t>(), n_adm, 64, s);
            partner_kernel<<<grid_for(n_adm), 256, 0, s>>>(tr->adm.as<int32_t>(), n_adm, k2.as<uint64_t>(),
                                                           i2.as<int32_t>(), tr->adm_tp.as<int32_t>());
            HM_LAUNCH_CHECK();
        }
    }

    // upper bound on touching pairs: sum over vertices of valence^2
    {
        DBuf val, sq;
        val.alloc(sizeof(int32_t) * nv);
        sq.alloc(sizeof(int64_t) * (nv + 1));
        HM_CUDA_CHECK(cudaMemsetAsync(val.p, 0, sizeof(int32_t) * nv, s));
        valence_kernel<<<grid_for(3 * n), 256, 0, s>>>(T.as<int32_t>(), n, val.as<int32_t>());
        HM_LAUNCH_CHECK();
        square_kernel<<<grid_for(nv), 256, 0, s>>>(val.as<int32_t>(), nv, sq.as<int64_t>());
        HM_LAUNCH_CHECK();
        tr->singular_cap = exclusive_scan_i64(sq.as<int64_t>(), sq.as<int64_t>(), nv, s);
    }

    // TMA descriptor of the panel table: box = [PT_ROWS][box_cols], box_cols
    // even and >= the largest dense dimension + 1 (a box starts at an even
    // column so that its first byte is 16-byte aligned)
    tr->box_cols = (tr->max_dense_dim + 1 + 1) / 2 * 2;
    if (tr->box_cols > 256) fail(HM_EINVAL, "leaf_size too large for the panel staging box");
    make_tensor_map_2d_f64(&tr->pt_map, tr->pt.as<double>(), (uint64_t)npad, PT_ROWS, (uint32_t)tr->box_cols,
                           PT_ROWS);
    // and of the float-pair table: box [PF_ROWS][box_cols_f], starting at a
    // column that is a multiple of 4 (0 = too wide: the FP64 entries are used)
    tr->box_cols_f = (tr->max_dense_dim + 3 + 3) / 4 * 4;
    if (tr->box_cols_f <= 256)
        make_tensor_map_2d_f32(&tr->pf_map, tr->pf.as<float>(), (uint64_t)npad, PF_ROWS, (uint32_t)tr->box_cols_f,
                               PF_ROWS);
    else
        tr->box_cols_f = 0;
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
    tr->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return tr.release();
}

}  // namespace hm
