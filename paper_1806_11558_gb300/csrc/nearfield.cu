// nearfield.cu -- dense (non-admissible) leaves of the block tree.
//
// Sec. 3.3 "Pre-computation of matrix blocks": every entry of every
// non-admissible leaf is evaluated once and stored contiguously without
// padding.  Here the storage unit is the row panel of a leaf row cluster (all
// dense blocks of that block row side by side), which is what the
// row-owned H-matrix-vector product streams.
//
// nearfield_kernel: one CTA per dense block (of a pair of blocks with swapped
// ranges, only the one above the diagonal works and writes both, the matrix
// being symmetric).  One elected thread stages the
// row cluster's and the column cluster's panel records (7 quadrature points,
// area, vertex ids) into shared memory with two 2-D TMA box loads completing
// on an mbarrier; every thread then evaluates entries with the 7x7 rule.
// Pairs that share a vertex are queued (warp-aggregated append) for
// singular_kernel, which gives each such entry one warp: the lanes split the
// Gauss points of the regularised integral.
#include "entry.cuh"
#include "ff.cuh"

namespace hm {

struct SingularItem {
    int64_t off;   // arena offset of the entry
    int64_t off2;  // arena offset of the transposed entry that receives the same value, or -1
    int32_t i;     // Morton row
    int32_t j;     // Morton column
};

// ---------------------------------------------------------------------------
// TMA / mbarrier (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
        : "memory");
}

// Bounded wait: gives up after `limit` SM clock cycles (sets *err), so a lost
// transaction can never hang the GPU.  The limit is checked before each poll:
// a limit of 0 gives up without polling (the test hook of hm_set_wait_limit).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, int *err, int code,
                                                  long long limit) {
    const long long t0 = clock64();
    for (;;) {
        if (clock64() - t0 >= limit) {
            atomicExch(err, code);
            return false;
        }
        if (mbar_try_wait(bar, phase)) return true;
    }
}

// Shared-memory layout of nearfield_kernel: two 128-byte aligned panel tiles
// (FP64: [PT_ROWS][box_cols] doubles; float pairs: [PF_ROWS][box_cols]
// floats), then the mbarrier.
__host__ __device__ constexpr int nf_rec_bytes(bool ff) { return ff ? PF_ROWS * 4 : PT_ROWS * 8; }
__host__ __device__ constexpr int nf_tile_bytes(bool ff, int box_cols) {
    return ((nf_rec_bytes(ff) * box_cols) + 127) / 128 * 128;
}
__host__ __device__ constexpr int nf_smem_bytes(bool ff, int box_cols) {
    return 128 + 2 * nf_tile_bytes(ff, box_cols) + 16;
}

// ---------------------------------------------------------------------------
// regular near-field entries
// ---------------------------------------------------------------------------
constexpr int NF_THREADS = 128;

// FF: the regular entries from the float-pair table in double-float
// arithmetic (regular_entry_ff, ~1e-14 relative) on the FP32 pipes; else from
// the FP64 table in FP64.
template <bool FF>
__global__ void __launch_bounds__(NF_THREADS) nearfield_kernel(const __grid_constant__ CUtensorMap pt_map,
                                                                const int32_t *__restrict__ dense,
                                                                const int64_t *__restrict__ base,
                                                                const int32_t *__restrict__ ld,
                                                                const int32_t *__restrict__ tp, int box_cols,
                                                                const QuadParams qp, double *__restrict__ arena,
                                                                SingularItem *__restrict__ sing,
                                                                unsigned long long *sing_count, int64_t sing_cap,
                                                                int *err, long long wait_limit) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int64_t b = blockIdx.x;
    const int32_t rb = dense[4 * b], re = dense[4 * b + 1], cb = dense[4 * b + 2], ce = dense[4 * b + 3];
    // the matrix is symmetric: of a pair of leaves with swapped ranges the one
    // above the diagonal evaluates the regular entries and stores them in
    // both; the one below has nothing to do
    const int32_t partner = tp[b];
    const bool mirror = partner >= 0 && partner != b;
    if (mirror && rb > cb) return;
    // a box starts at a column whose first byte is 16-byte aligned
    const int32_t rb_al = FF ? rb & ~3 : rb & ~1, cb_al = FF ? cb & ~3 : cb & ~1;
    const int tile_bytes = nf_tile_bytes(FF, box_cols);
    using Rec = typename std::conditional<FF, float, double>::type;
    Rec *tR = reinterpret_cast<Rec *>(sm);
    Rec *tC = reinterpret_cast<Rec *>(sm + tile_bytes);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * tile_bytes);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, 2u * (uint32_t)nf_rec_bytes(FF) * box_cols);
        tma_load_2d(tR, &pt_map, bar, rb_al, 0);
        tma_load_2d(tC, &pt_map, bar, cb_al, 0);
    }
    if (!mbar_wait_bounded(bar, 0, err, 2, wait_limit)) {
        // the copies this block started may still land in its shared memory:
        // wait for them (with the default bound) before leaving
        mbar_wait_bounded(bar, 0, err, 2, WAIT_LIMIT_DEFAULT);
        return;
    }
    const int m = re - rb, n = ce - cb, mn = m * n;
    const int ro = rb - rb_al, co = cb - cb_al;
    const int64_t blk_base = base[b];
    const int32_t blk_ld = ld[b];
    const int64_t par_base = mirror ? base[partner] : 0;
    const int32_t par_ld = mirror ? ld[partner] : 0;
    const int lane = threadIdx.x & 31;
    for (int e0 = 0; e0 < mn; e0 += NF_THREADS) {
        const int e = e0 + threadIdx.x;
        const bool valid = e < mn;
        const int i = valid ? e / n : 0, j = valid ? e - (e / n) * n : 0;
        const Rec *R = tR + i + ro;
        const Rec *C = tC + j + co;
        int32_t vr[3], vc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if constexpr (FF) {
                vr[k] = __float_as_int(R[(PF_VID + k) * box_cols]);
                vc[k] = __float_as_int(C[(PF_VID + k) * box_cols]);
            } else {
                vr[k] = (int32_t)R[(PT_VID + k) * box_cols];
                vc[k] = (int32_t)C[(PT_VID + k) * box_cols];
            }
        }
        const int kind = valid ? shared_vertices(vr, vc) : 0;
        const bool touch = kind > 0;
        // Touching pairs go to the Sauter-Schwab queue.  A common-edge pair is
        // evaluated in both orientations: the regularised rule depends on
        // which panel comes first, by up to ~1e-10 at n_ss = 8.  A
        // common-vertex pair gives the same value in both orientations up to
        // rounding (the two regions are mirror images), so it is evaluated
        // once and stored at (i, j) and (j, i): by the upper block of a
        // mirrored pair, or inside a diagonal block by the entry with i < j.
        const bool diag = partner == b;
        const bool once = kind == 1 && (mirror || diag);
        const bool skip = once && diag && i > j;
        const int per = !touch || skip ? 0 : (mirror && !once) ? 2 : 1;
        const unsigned b1 = __ballot_sync(0xffffffffu, per == 1), b2 = __ballot_sync(0xffffffffu, per == 2);
        if (b1 | b2) {
            const int leader = __ffs(b1 | b2) - 1;
            unsigned long long slot = 0;
            if (lane == leader) slot = atomicAdd(sing_count, (unsigned long long)(__popc(b1) + 2 * __popc(b2)));
            slot = __shfl_sync(0xffffffffu, slot, leader);
            if (per > 0) {
                const unsigned lower = (1u << lane) - 1u;
                const unsigned long long k = slot + __popc(b1 & lower) + 2 * __popc(b2 & lower);
                if ((int64_t)k + per <= sing_cap) {
                    const int64_t off_t = mirror ? par_base + (int64_t)j * par_ld + i
                                                 : blk_base + (int64_t)j * blk_ld + i;
                    sing[k].off = blk_base + (int64_t)i * blk_ld + j;
                    sing[k].off2 = once ? off_t : -1;
                    sing[k].i = rb + i;
                    sing[k].j = cb + j;
                    if (per == 2) {
                        sing[k + 1].off = off_t;
                        sing[k + 1].off2 = -1;
                        sing[k + 1].i = cb + j;
                        sing[k + 1].j = rb + i;
                    }
                } else {
                    atomicExch(err, 3);
                }
            }
        }
        if (valid && !touch) {
            double a;
            if constexpr (FF)
                a = regular_entry_ff(R, box_cols, C, box_cols, qp.w_h, qp.w_l);
            else
                a = regular_entry(R, box_cols, C, box_cols, qp);
            arena[blk_base + (int64_t)i * blk_ld + j] = a;
            if (mirror) arena[par_base + (int64_t)j * par_ld + i] = a;
        }
    }
}

// ---------------------------------------------------------------------------
// touching pairs: one warp per entry
//
// The rule is the tensor Gauss-Legendre rule in (eta1, eta2, eta3) over the
// Sauter-Schwab regions (entry.cuh).  For flat panels part of each integrand
// is a low-degree polynomial that an n-point Gauss rule integrates exactly,
// so the same rule value needs fewer evaluations:
//  * identical panels: chi(u) - chi(v) = J (u - v) and in every region
//    u - v = eta1 eta2 d(eta3) while the Jacobian is eta1^2 eta2, so the
//    integrand is eta1 / |J d(eta3)|: the eta1 and eta2 sums are exactly 1/2
//    and 1, the six regions pair up, and the value is
//    sum_k w_k [1/|J(e_k,1)| + 1/|J(1,e_k)| + 1/|J(-e_k,1-e_k)|];
//  * common edge: D = eta1 D'(eta2, eta3) and Jacobian = eta1^2 j'(eta2), so
//    the eta1 sum is exactly 1/2 and a 2-D sum remains;
//  * common vertex: the full 3-D sum.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double inv_norm3(double x, double y, double z) { return rsqrt(fma(x, x, fma(y, y, z * z))); }

// Common-vertex and common-edge rules in double-float arithmetic.  The 2 n^3
// points of the two common-vertex regions (and the 5 n^2 of the common-edge
// 2-D sum) are tabulated once per assembly (FP64 values split into float
// pairs): the coefficients (u0, u1, v0, v1) of D = (u0 a1 + u1 a2) -
// (v0 b1 + v1 b2) and the weight w1 w2 w3 * jac.  Per point the products of
// the coefficients with the edge vectors are exact (TwoProduct) up to the
// float-pair rounding of the inputs, their high parts add exactly (TwoSum)
// and every low part goes to one float, so D is accurate to about 2^-48 of
// its largest term, as in FP64 up to the shorter mantissa.
struct SSPointFF {
    float ch[4], cl[4];  // u0, u1, v0, v1
    float wh, wl;        // w1 w2 w3 jac
};

__global__ void ss_vertex_table_kernel(const QuadParams qp, SSPointFF *tab) {
    const int n = qp.ss_n, n3 = n * n * n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * n3; t += gridDim.x * blockDim.x) {
        const int r = t / n3, rem = t - r * n3;
        const int k1 = rem / (n * n), k2 = (rem / n) % n, k3 = rem % n;
        double c[4], jac;
        ss_region(1, r, qp.gx[k1], qp.gx[k2], qp.gx[k3], c[0], c[1], c[2], c[3], jac);
        SSPointFF p;
        for (int k = 0; k < 4; ++k) split_double(c[k], p.ch[k], p.cl[k]);
        split_double(qp.gw[k1] * qp.gw[k2] * qp.gw[k3] * jac, p.wh, p.wl);
        tab[t] = p;
    }
}

// The common-edge rule after the exact eta1 sum (the 2-D sum of the FP64
// path below): D' = d0 a1 + u1 a2 - v1 b2 over the five regions, weight
// w2 w3 jp / 2, stored as coefficients of (a1, a2, b2, b1) with the last 0.
__global__ void ss_edge_table_kernel(const QuadParams qp, SSPointFF *tab) {
    const int n = qp.ss_n, n2 = n * n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 5 * n2; t += gridDim.x * blockDim.x) {
        const int r = t / n2, rem = t - r * n2, k2 = rem / n, k3 = rem - k2 * n;
        const double e2 = qp.gx[k2], e3 = qp.gx[k3], e23 = e2 * e3;
        double d0, u1, v1, jp;
        switch (r) {
            case 0: d0 = e2; u1 = e3; v1 = 1.0 - e2; jp = 1.0; break;
            case 1: d0 = e23; u1 = 1.0; v1 = e2 - e23; jp = e2; break;
            case 2: d0 = -e2; u1 = 1.0 - e2; v1 = e23; jp = e2; break;
            case 3: d0 = -e23; u1 = e2 - e23; v1 = 1.0; jp = e2; break;
            default: d0 = -e23; u1 = 1.0 - e23; v1 = e2; jp = e2; break;
        }
        SSPointFF p;
        const double c[4] = {d0, u1, v1, 0.0};
        for (int k = 0; k < 4; ++k) split_double(c[k], p.ch[k], p.cl[k]);
        split_double(0.5 * (qp.gw[k2] * qp.gw[k3] * jp), p.wh, p.wl);
        tab[t] = p;
    }
}

// (s, e) += (a, b) for non-negative float pairs
__device__ __forceinline__ void ff_acc(float &s, float &e, float a, float b) {
    float t, u;
    two_sum(s, a, t, u);
    s = t;
    e = __fadd_rn(e, __fadd_rn(u, b));
}

// Sum over this lane's points of w / |D|, D = c0 E0 + c1 E1 - c2 E2 - c3 E3,
// for the edge vectors E (common vertex: (a1, a2, b1, b2); common edge:
// (a1, a2, b2, b1) with c3 = 0) as float pairs; returned as a float pair.
__device__ __forceinline__ void ss_sum_ff(const float Eh[4][3], const float El[4][3], const SSPointFF *__restrict__ tab,
                                             int npts, int lane, float &acc_h, float &acc_l) {
    acc_h = 0.0f;
    acc_l = 0.0f;
    for (int t = lane; t < npts; t += 32) {
        const SSPointFF p = tab[t];
        float dd_h = 0.0f, dd_l = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            // D_d = c0 a1 + c1 a2 - c2 b1 - c3 b2
            float hs = 0.0f, lo = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float sg = k < 2 ? 1.0f : -1.0f;
                float ph, pe;
                two_prod(p.ch[k], Eh[k][d], ph, pe);
                pe = __fmaf_rn(p.ch[k], El[k][d], pe);
                pe = __fmaf_rn(p.cl[k], Eh[k][d], pe);
                float t1, e1;
                two_sum(hs, sg * ph, t1, e1);
                hs = t1;
                lo = __fadd_rn(lo, __fmaf_rn(sg, pe, e1));
            }
            float Dh, Dl;
            fast_two_sum(hs, lo, Dh, Dl);
            // dd += D^2
            float qh, ql;
            two_prod(Dh, Dh, qh, ql);
            ql = __fmaf_rn(__fmul_rn(2.0f, Dh), Dl, ql);
            ff_acc(dd_h, dd_l, qh, ql);
        }
        float r2h, r2l;
        fast_two_sum(dd_h, dd_l, r2h, r2l);
        // 1 / sqrt(r2): estimate + one Newton step with an exact residual
        const float y0 = rsqrtf(r2h);
        float yh, yl;
        two_prod(y0, y0, yh, yl);
        float mh, ml;
        two_prod(r2h, yh, mh, ml);
        ml = __fmaf_rn(r2h, yl, ml);
        ml = __fmaf_rn(r2l, yh, ml);
        const float del = __fsub_rn(__fsub_rn(1.0f, mh), ml);
        const float corr = __fmul_rn(__fmul_rn(0.5f, y0), del);
        // acc += w (y0 + corr)
        float qh, ql;
        two_prod(p.wh, y0, qh, ql);
        ql = __fmaf_rn(p.wh, corr, ql);
        ql = __fmaf_rn(p.wl, y0, ql);
        ff_acc(acc_h, acc_l, qh, ql);
    }
}

__global__ void singular_kernel(const SingularItem *__restrict__ items, int64_t count, const int32_t *__restrict__ trim,
                                const double *__restrict__ V, const double *__restrict__ pt, int64_t npad,
                                const QuadParams qp, double *__restrict__ arena,
                                const SSPointFF *__restrict__ vtab, const SSPointFF *__restrict__ etab) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= count) return;
    const SingularItem it = items[w];
    const int32_t *ta = trim + 3 * (int64_t)it.i, *tb = trim + 3 * (int64_t)it.j;
    const int32_t a[3] = {ta[0], ta[1], ta[2]}, bb[3] = {tb[0], tb[1], tb[2]};
    const int kind = shared_vertices(a, bb);
    int32_t P[3], Q[3];
    touch_orient(a, bb, kind, P, Q);
    const PairGeom g = pair_geom(V, P, Q);
    const int n = qp.ss_n, n2 = n * n, n3 = n2 * n;
    double s = 0.0;
    bool ff_done = false;
    if (kind == 3) {
        // 1-D: three classes of regions, each counted twice with the eta1 / eta2 sums 1/2 and 1
        for (int t = lane; t < 3 * n; t += 32) {
            const int c = t / n, k = t - c * n;
            const double e = qp.gx[k];
            double s0, s1;
            if (c == 0) { s0 = e; s1 = 1.0; }
            else if (c == 1) { s0 = 1.0; s1 = e; }
            else { s0 = -e; s1 = 1.0 - e; }
            s += qp.gw[k] * inv_norm3(s0 * g.a1[0] + s1 * g.a2[0], s0 * g.a1[1] + s1 * g.a2[1],
                                      s0 * g.a1[2] + s1 * g.a2[2]);
        }
    } else if (kind != 3 && (kind == 1 ? vtab : etab)) {
        // double-float points; the lanes' partial sums as float pairs
        float Eh[4][3], El[4][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            split_double(g.a1[d], Eh[0][d], El[0][d]);
            split_double(g.a2[d], Eh[1][d], El[1][d]);
            split_double(kind == 1 ? g.b1[d] : g.b2[d], Eh[2][d], El[2][d]);
            split_double(kind == 1 ? g.b2[d] : g.b1[d], Eh[3][d], El[3][d]);
        }
        float ah, al;
        ss_sum_ff(Eh, El, kind == 1 ? vtab : etab, kind == 1 ? 2 * n3 : 5 * n2, lane, ah, al);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, ah, o), bl = __shfl_xor_sync(0xffffffffu, al, o);
            ff_acc(ah, al, bh, bl);
        }
        s = (double)ah + (double)al;  // the same value on every lane
        ff_done = true;
    } else if (kind == 2) {
        // 2-D: D' = d0 a1 + u1 a2 - v1 b2 over the five regions, eta1 sum = 1/2
        for (int t = lane; t < 5 * n2; t += 32) {
            const int r = t / n2, rem = t - r * n2, k2 = rem / n, k3 = rem - k2 * n;
            const double e2 = qp.gx[k2], e3 = qp.gx[k3], e23 = e2 * e3;
            double d0, u1, v1, jp;
            switch (r) {
                case 0: d0 = e2; u1 = e3; v1 = 1.0 - e2; jp = 1.0; break;
                case 1: d0 = e23; u1 = 1.0; v1 = e2 - e23; jp = e2; break;
                case 2: d0 = -e2; u1 = 1.0 - e2; v1 = e23; jp = e2; break;
                case 3: d0 = -e23; u1 = e2 - e23; v1 = 1.0; jp = e2; break;
                default: d0 = -e23; u1 = 1.0 - e23; v1 = e2; jp = e2; break;
            }
            const double dx = d0 * g.a1[0] + u1 * g.a2[0] - v1 * g.b2[0];
            const double dy = d0 * g.a1[1] + u1 * g.a2[1] - v1 * g.b2[1];
            const double dz = d0 * g.a1[2] + u1 * g.a2[2] - v1 * g.b2[2];
            s += qp.gw[k2] * qp.gw[k3] * jp * inv_norm3(dx, dy, dz);
        }
        s *= 0.5;
    } else {
        for (int t = lane; t < 2 * n3; t += 32) {
            const int r = t / n3, rem = t - r * n3;
            const int k1 = rem / n2, k2 = (rem / n) % n, k3 = rem % n;
            s += ss_point(g, kind, r, k1, k2, k3, qp);
        }
    }
    if (!ff_done) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0) {
        const double ai = pt[(int64_t)PT_AREA * npad + it.i], aj = pt[(int64_t)PT_AREA * npad + it.j];
        const double a = 4.0 * ai * aj * (s / 3.0) * INV_4PI;
        arena[it.off] = a;
        if (it.off2 >= 0) arena[it.off2] = a;
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
void assemble_nearfield(const hm_tree *tr, hm_matrix *A, const QuadParams &qp, cudaStream_t s, int *d_err,
                        double *sec_regular, double *sec_singular, bool fp64) {
    // padding columns of the row panels must read as 0
    A->dense.alloc(sizeof(double) * std::max<int64_t>(tr->dense_entries, 1));
    HM_CUDA_CHECK(cudaMemsetAsync(A->dense.p, 0, sizeof(double) * std::max<int64_t>(tr->dense_entries, 1), s));
    DBuf items, cnt;
    items.alloc(sizeof(SingularItem) * std::max<int64_t>(tr->singular_cap, 1));
    cnt.alloc(sizeof(unsigned long long));
    HM_CUDA_CHECK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s));
    const bool ff = !fp64 && tr->box_cols_f > 0;
    const int box = ff ? tr->box_cols_f : tr->box_cols;
    const int smem = nf_smem_bytes(ff, box);
    auto kern = ff ? nearfield_kernel<true> : nearfield_kernel<false>;
    HM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    cudaEvent_t e0, e1, e2;
    HM_CUDA_CHECK(cudaEventCreate(&e0));
    HM_CUDA_CHECK(cudaEventCreate(&e1));
    HM_CUDA_CHECK(cudaEventCreate(&e2));
    HM_CUDA_CHECK(cudaEventRecord(e0, s));
    if (tr->n_dense > 0) {
        Trace trace(ff ? "nearfield_kernel" : "nearfield_kernel.f64", s);
        kern<<<(unsigned)tr->n_dense, NF_THREADS, smem, s>>>(
            ff ? tr->pf_map : tr->pt_map, tr->dense.as<int32_t>(), tr->dense_base.as<int64_t>(),
            tr->dense_ld.as<int32_t>(), tr->dense_tp.as<int32_t>(), box, qp, A->dense.as<double>(),
            items.as<SingularItem>(), cnt.as<unsigned long long>(), tr->singular_cap, d_err, wait_limit());
        HM_LAUNCH_CHECK();
    }
    HM_CUDA_CHECK(cudaEventRecord(e1, s));
    const int64_t nsing = (int64_t)read_scalar(cnt.as<unsigned long long>(), s);
    if (nsing > tr->singular_cap) fail(HM_EINTERNAL, "touching-pair queue overflow (%lld > %lld)", (long long)nsing,
                                      (long long)tr->singular_cap);
    const_cast<hm_tree *>(tr)->n_singular = nsing;
    DBuf vtab;  // freed after the synchronisation below
    if (nsing > 0) {
        // common-vertex pairs in double-float unless FP64 entries were asked for
        if (!fp64) {
            const int nv = 2 * qp.ss_n * qp.ss_n * qp.ss_n, ne = 5 * qp.ss_n * qp.ss_n;
            vtab.alloc(sizeof(SSPointFF) * (nv + ne));
            ss_vertex_table_kernel<<<(nv + 255) / 256, 256, 0, s>>>(qp, vtab.as<SSPointFF>());
            HM_LAUNCH_CHECK();
            ss_edge_table_kernel<<<(ne + 255) / 256, 256, 0, s>>>(qp, vtab.as<SSPointFF>() + nv);
            HM_LAUNCH_CHECK();
        }
        const int64_t threads = nsing * 32;
        Trace trace("singular_kernel", s);
        singular_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
            items.as<SingularItem>(), nsing, tr->trim.as<int32_t>(), tr->V.as<double>(), tr->pt.as<double>(),
            tr->npad, qp, A->dense.as<double>(), vtab.as<SSPointFF>(),
            vtab.p ? vtab.as<SSPointFF>() + 2 * qp.ss_n * qp.ss_n * qp.ss_n : nullptr);
        HM_LAUNCH_CHECK();
    }
    HM_CUDA_CHECK(cudaEventRecord(e2, s));
    HM_CUDA_CHECK(cudaEventSynchronize(e2));
    float ms1 = 0, ms2 = 0;
    HM_CUDA_CHECK(cudaEventElapsedTime(&ms1, e0, e1));
    HM_CUDA_CHECK(cudaEventElapsedTime(&ms2, e1, e2));
    *sec_regular = ms1 * 1e-3;
    *sec_singular = ms2 * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
}

}  // namespace hm
