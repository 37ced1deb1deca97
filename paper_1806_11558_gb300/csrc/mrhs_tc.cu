// mrhs_tc.cu -- the row pass of the 16-right-hand-side H-matrix product
// (Sec. 2.3, the near-field and U panels of every leaf row cluster against
// the gathered rows of X and t) on the fifth-generation tensor cores:
// tcgen05.mma with the accumulator in tensor memory (TMEM).
//
//   D (rows x 32, FP32, TMEM) = A_hi B + [A_lo B_hi | 0],   B = [Z_hi | Z_lo]
//
// A is a slice of 64 panel columns, split into BF16 hi / lo planes (FP32
// panels) or taken as it is (BF16 factors); B holds the gathered rows of X
// (or t) as BF16 pairs, 16 hi and 16 lo columns.  The three products
// hi*hi, hi*lo, lo*hi of the mma.sync kernel are two MMAs here (N = 32 and
// N = 16); the epilogue adds the two halves of D.
//
// One CTA of 128 threads per leaf row cluster (and 128-row tile).  Per slice:
// the threads load the panel rows with coalesced 16-byte loads one slice
// ahead into registers, split them and store both planes into shared memory
// in the canonical K-major layout without swizzle (8 x 16-byte core
// matrices); the gathered rows of B land by cp.async, one slice ahead, in the
// MN-major layout; one thread issues the MMAs of the slice and commits them
// to the slice buffer's mbarrier, which the threads wait on before they
// overwrite that buffer two slices later.  Every wait is bounded
// (hm_set_wait_limit): a wait that gives up records an error code, waits for
// its B copies and (bounded by the default limit) for the MMAs it issued,
// frees the tensor memory and leaves the CTA.
#include <cuda_bf16.h>

#include <algorithm>

#include "hm_internal.cuh"

namespace hm {
namespace tc {

constexpr int THREADS = 128;
constexpr int KS = 64;                        // panel columns per slice
constexpr int NB = 32;                        // B columns: 16 hi, 16 lo
constexpr int B_SBO = 128;                    // bytes between N-adjacent core matrices of B
constexpr int B_LBO = NB / 8 * 128;           // bytes between K-adjacent core matrices of B (512)
constexpr int B_BYTES = KS / 8 * B_LBO;       // 4 KB per slice
constexpr int B_RING = 3;                     // B is gathered one slice ahead
constexpr int A_SBO = 128;                    // bytes between M-adjacent core matrices of A
constexpr int TMEM_COLS = 32;

__host__ __device__ constexpr int a_lbo(int arows) { return arows * 16; }      // K-adjacent core matrices
__host__ __device__ constexpr int a_plane(int arows) { return KS / 8 * a_lbo(arows); }
// shared memory: [2 stages][hi, lo planes], [B_RING][B], barriers + TMEM address, then
// padding that the 128-row MMA reads past the last plane when arows < 128
__host__ __device__ constexpr int smem_bytes(int arows) {
    return 2 * 2 * a_plane(arows) + B_RING * B_BYTES + 64 + 2048 + 128;
}

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, start / leading / stride byte offsets
__device__ __forceinline__ uint64_t desc(uint32_t start, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((start & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, A K-major, B MN-major, M = 128
__host__ __device__ constexpr uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ bool try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded by `limit` SM clock cycles (try_wait itself may suspend for a
// while); a limit of 0 gives up without polling (hm_set_wait_limit)
__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        if (clock64() - t0 >= limit) return false;
        if (try_wait(bar, parity)) return true;
    }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void cp16(void *dst, const void *src, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr(dst)), "l"(src), "r"(pred ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t pack(float lo_k, float hi_k) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Four consecutive panel values (16 bytes of FP32, 8 bytes of BF16): one
// unit of the per-slice load; `u` indexes (row group of 8, column block of
// 16) and the lane its (row, 4 columns) in them.
template <class TP> struct Quad;
template <> struct Quad<float> {
    float4 v;
    __device__ __forceinline__ void load(const float *p, bool ok) {
        v = ok ? __ldg(reinterpret_cast<const float4 *>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // hi / lo planes: 4 BF16 each (8 bytes)
    __device__ __forceinline__ void store(unsigned char *hi, unsigned char *lo, int off) const {
        const float a[4] = {v.x, v.y, v.z, v.w};
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = __bfloat162float(__float2bfloat16_rn(a[e]));
            l[e] = a[e] - h[e];
        }
        *reinterpret_cast<uint2 *>(hi + off) = make_uint2(pack(h[0], h[1]), pack(h[2], h[3]));
        *reinterpret_cast<uint2 *>(lo + off) = make_uint2(pack(l[0], l[1]), pack(l[2], l[3]));
    }
};
template <> struct Quad<__nv_bfloat16> {
    uint2 v;
    __device__ __forceinline__ void load(const __nv_bfloat16 *p, bool ok) {
        v = ok ? __ldg(reinterpret_cast<const uint2 *>(p)) : make_uint2(0u, 0u);
    }
    __device__ __forceinline__ void store(unsigned char *hi, unsigned char *, int off) const {
        *reinterpret_cast<uint2 *>(hi + off) = v;
    }
};

// A slice in flight: the units of this thread (warp w takes units w, w + 4,
// ...): U per thread covers tiles of 8 U rows (4 column blocks x 8 U / 8 row
// groups over 4 warps)
template <class TP, int U> struct Slice {
    Quad<TP> q[U];
};

// Panel source of one pass: rows [r0t, r0t + rows) of a row-major panel of K
// columns, gathered rows Zh / Zl (BF16 pairs, [row][16]) by idx.
template <class TP> struct Src {
    const TP *P;
    int K;
    const int32_t *idx;
    const __nv_bfloat16 *Zh, *Zl;
};

template <class TP, int U>
__device__ __forceinline__ void load_slice(Slice<TP, U> &sl, const Src<TP> &s, int rows, int k0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nunits = (rows + 7) / 8 * (KS / 16);
#pragma unroll
    for (int i = 0; i < U; ++i) {
        const int u = warp + 4 * i;
        const int r = 8 * (u >> 2) + (lane & 7), k = k0 + 16 * (u & 3) + 4 * (lane >> 3);
        const bool ok = u < nunits && r < rows && k < s.K;
        sl.q[i].load(s.P + (ok ? (int64_t)r * s.K + k : 0), ok);
    }
}

// the units of a slice into the two A planes (K-major core matrices)
template <class TP, int U>
__device__ __forceinline__ void store_slice(const Slice<TP, U> &sl, unsigned char *hi, unsigned char *lo, int rows,
                                            int arows) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nunits = (rows + 7) / 8 * (KS / 16);
#pragma unroll
    for (int i = 0; i < U; ++i) {
        const int u = warp + 4 * i;
        const int r = 8 * (u >> 2) + (lane & 7), kl = 16 * (u & 3) + 4 * (lane >> 3);
        if (u < nunits && r < rows) {
            const int off = (kl >> 3) * a_lbo(arows) + (r >> 3) * A_SBO + (r & 7) * 16 + (kl & 7) * 2;
            sl.q[i].store(hi, lo, off);
        }
    }
}

// the gathered rows of B for the slice at k0 (zero beyond K), MN-major core matrices
template <class TP>
__device__ __forceinline__ void gather_b(unsigned char *b, const Src<TP> &s, int k0) {
    for (int p = threadIdx.x; p < 4 * KS; p += THREADS) {
        const int q = p / KS, kk = p - q * KS;  // q: hi n 0-7, hi n 8-15, lo n 0-7, lo n 8-15
        const int col = k0 + kk;
        const bool ok = col < s.K;
        const int row = ok ? __ldg(s.idx + col) : 0;
        const __nv_bfloat16 *src = ((q & 2) ? s.Zl : s.Zh) + (int64_t)row * 16 + 8 * (q & 1);
        cp16(b + q * B_SBO + (kk >> 3) * B_LBO + (kk & 7) * 16, src, ok);
    }
    cp_commit();
}

struct Ctx {
    unsigned char *a;    // [2 stages][hi plane, lo plane]
    unsigned char *b;    // [B_RING] slices of B
    uint64_t *bar;       // [2] MMA completion of the slices in each stage
    uint32_t tmem;       // D
    int arows;
    long long slice;     // slices issued by this CTA so far
    long long limit;     // bound of the waits (SM clock cycles)
    bool first;          // the next MMA starts the tile's accumulation
    bool failed;
};

// One panel of the tile through the pipeline (FP32 panels: split == true).
template <class TP, int U>
__device__ bool run_panel(Ctx &c, const Src<TP> &s, int rows, int *err) {
    constexpr bool split = sizeof(TP) == 4;
    const int ns = (s.K + KS - 1) / KS;
    if (ns == 0) return true;
    const int plane = a_plane(c.arows);
    // panel slices are loaded one slice ahead of their conversion (registers;
    // two ahead measured slower: 168 registers with spills, 17.7 against
    // 15.4 ms per level-8 row pass)
    Slice<TP, U> cur;
    load_slice(cur, s, rows, 0);
    gather_b(c.b + (c.slice % B_RING) * B_BYTES, s, 0);
    for (int k = 0; k < ns; ++k) {
        const long long sidx = c.slice + k;
        const int st = (int)(sidx & 1);
        unsigned char *hi = c.a + st * 2 * plane, *lo = hi + plane;
        unsigned char *bb = c.b + (sidx % B_RING) * B_BYTES;
        // the stage's previous slice (sidx - 2) must be consumed by its MMAs
        const bool ok = sidx < 2 || wait(c.bar + st, (uint32_t)(((sidx >> 1) - 1) & 1), c.limit);
        if (ok) store_slice(cur, hi, lo, rows, c.arows);
        if (k + 1 < ns) {
            load_slice(cur, s, rows, (k + 1) * KS);  // registers: consumed next iteration
            gather_b(c.b + ((sidx + 1) % B_RING) * B_BYTES, s, (k + 1) * KS);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this slice's B landed
        } else {
            cp_wait_all();
        }
        fence_proxy();
        if (__syncthreads_or(!ok)) {  // a wait that gave up, seen by every thread alike
            cp_wait_all();            // the next slice's B may still be landing
            if (threadIdx.x == 0) atomicExch(err, 1);
            c.failed = true;
            c.slice += k;
            return false;
        }
        if (threadIdx.x == 0) {
            fence_after();
            const int ksteps = min(KS, s.K - k * KS + 15) / 16;
#pragma unroll 1
            for (int kk = 0; kk < ksteps; ++kk) {
                const uint64_t ad = desc(saddr(hi) + kk * 2 * a_lbo(c.arows), a_lbo(c.arows), A_SBO);
                const uint64_t bd = desc(saddr(bb) + kk * 2 * B_LBO, B_LBO, B_SBO);
                mma(c.tmem, ad, bd, idesc(32), c.first ? 0u : 1u);
                c.first = false;
                if (split) {
                    const uint64_t ld = desc(saddr(lo) + kk * 2 * a_lbo(c.arows), a_lbo(c.arows), A_SBO);
                    mma(c.tmem, ld, bd, idesc(16), 1u);
                }
            }
            commit(c.bar + st);
        }
        // keep `first` in step on every thread (only thread 0 issues)
        c.first = false;
    }
    c.slice += ns;
    return true;
}

template <class TF, int U>
__global__ void __launch_bounds__(THREADS, 3) row_mrhs_tc_kernel(
    const int32_t *__restrict__ leaf_begin, const int64_t *__restrict__ rho_off, const int32_t *__restrict__ rho_K,
    const int64_t *__restrict__ rho_colptr, const int32_t *__restrict__ colidx, const float *__restrict__ dense,
    const int64_t *__restrict__ up_off, const int32_t *__restrict__ up_K, const int64_t *__restrict__ up_colptr,
    const int32_t *__restrict__ tidx, const TF *__restrict__ up, const __nv_bfloat16 *__restrict__ Th,
    const __nv_bfloat16 *__restrict__ Tl, const __nv_bfloat16 *__restrict__ Xh, const __nv_bfloat16 *__restrict__ Xl,
    double *__restrict__ Y, int arows, int *err, long long wait_limit) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    Ctx c;
    c.arows = arows;
    c.limit = wait_limit;
    c.a = sm;
    c.b = sm + 4 * a_plane(arows);
    c.bar = reinterpret_cast<uint64_t *>(c.b + B_RING * B_BYTES);
    uint32_t *taddr = reinterpret_cast<uint32_t *>(c.bar + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(c.bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(c.bar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(taddr)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    c.tmem = *taddr;
    c.slice = 0;
    c.failed = false;
    const int64_t rho = blockIdx.x;
    const int32_t r0 = leaf_begin[rho], mr = leaf_begin[rho + 1] - r0;
    const int Kd = rho_K[rho], Ku = up_K[rho];
    for (int r0t = 0; r0t < mr && !c.failed; r0t += 8 * U) {
        const int rows = min(8 * U, mr - r0t);
        c.first = true;
        const Src<float> sd{dense + rho_off[rho] + (int64_t)r0t * Kd, Kd, colidx + rho_colptr[rho], Xh, Xl};
        const Src<TF> su{up + up_off[rho] + (int64_t)r0t * Ku, Ku, tidx + up_colptr[rho], Th, Tl};
        if (!run_panel<float, U>(c, sd, rows, err)) break;
        if (!run_panel<TF, U>(c, su, rows, err)) break;
        // the tile's last commit covers every MMA issued so far
        float d[32];
        const bool any = c.slice > 0;
        const bool ok =
            !any || wait(c.bar + (int)((c.slice - 1) & 1), (uint32_t)(((c.slice - 1) >> 1) & 1), c.limit);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            c.failed = true;
            break;
        }
        fence_after();
        const uint32_t ta = c.tmem + ((uint32_t)(32 * warp) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]), "=f"(d[4]), "=f"(d[5]), "=f"(d[6]), "=f"(d[7]),
              "=f"(d[8]), "=f"(d[9]), "=f"(d[10]), "=f"(d[11]), "=f"(d[12]), "=f"(d[13]), "=f"(d[14]), "=f"(d[15]),
              "=f"(d[16]), "=f"(d[17]), "=f"(d[18]), "=f"(d[19]), "=f"(d[20]), "=f"(d[21]), "=f"(d[22]),
              "=f"(d[23]), "=f"(d[24]), "=f"(d[25]), "=f"(d[26]), "=f"(d[27]), "=f"(d[28]), "=f"(d[29]),
              "=f"(d[30]), "=f"(d[31])
            : "r"(ta)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = 32 * warp + lane;
        if (row < rows) {
            double2 *y = reinterpret_cast<double2 *>(Y + (int64_t)(r0 + r0t + row) * 16);
#pragma unroll
            for (int e = 0; e < 8; ++e)
                y[e] = any ? make_double2((double)(d[2 * e] + d[16 + 2 * e]), (double)(d[2 * e + 1] + d[17 + 2 * e]))
                           : make_double2(0.0, 0.0);
        }
        // every thread's reads of D are done before the next tile's MMAs overwrite it
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (c.failed && c.slice > 0) {
        // wait (bounded) for the MMAs this CTA issued before the TMEM goes away
        wait(c.bar + (int)((c.slice - 1) & 1), (uint32_t)(((c.slice - 1) >> 1) & 1), WAIT_LIMIT_DEFAULT);
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace tc

// Host launcher of the tensor-memory row pass (same data as row_mrhs_kernel).
template <class TF>
void row_mrhs_tc(const hm_matrix *A, const TF *up, const __nv_bfloat16 *Th, const __nv_bfloat16 *Tl,
                 const __nv_bfloat16 *Xh, const __nv_bfloat16 *Xl, double *Y, int *err, cudaStream_t s) {
    const hm_tree *tr = A->tree;
    // rows per pass: the largest leaf cluster rounded up to 8, 40 / 80 / 128 (U = rows / 8 units per thread)
    const int arows = tr->max_leaf <= 40 ? 40 : tr->max_leaf <= 80 ? 80 : 128;
    const int smem = tc::smem_bytes(arows);
    auto kern = arows == 40 ? tc::row_mrhs_tc_kernel<TF, 5>
                            : arows == 80 ? tc::row_mrhs_tc_kernel<TF, 10> : tc::row_mrhs_tc_kernel<TF, 16>;
    HM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    Trace trace(sizeof(TF) == 4 ? "row_mrhs_kernel.f32" : "row_mrhs_kernel.bf16", s);
    kern<<<(unsigned)tr->n_leaf, tc::THREADS, smem, s>>>(
        tr->leaf_begin.as<int32_t>(), tr->rho_off.as<int64_t>(), tr->rho_K.as<int32_t>(), tr->rho_colptr.as<int64_t>(),
        tr->colidx.as<int32_t>(), A->dense32.as<float>(), A->up_off.as<int64_t>(), A->up_K.as<int32_t>(),
        A->up_colptr.as<int64_t>(), A->tidx.as<int32_t>(), up, Th, Tl, Xh, Xl, Y, arows, err, wait_limit());
    HM_LAUNCH_CHECK();
}

template void row_mrhs_tc<float>(const hm_matrix *, const float *, const __nv_bfloat16 *, const __nv_bfloat16 *,
                                 const __nv_bfloat16 *, const __nv_bfloat16 *, double *, int *, cudaStream_t);
template void row_mrhs_tc<__nv_bfloat16>(const hm_matrix *, const __nv_bfloat16 *, const __nv_bfloat16 *,
                                         const __nv_bfloat16 *, const __nv_bfloat16 *, const __nv_bfloat16 *,
                                         double *, int *, cudaStream_t);

}  // namespace hm
