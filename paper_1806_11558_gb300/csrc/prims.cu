// prims.cu -- errors, device buffers, quadrature constants, scan, radix sort,
// TMA descriptors.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <map>
#include <mutex>

#include "hm_internal.cuh"

namespace hm {

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

const char *last_error_cstr() { return g_last_error.c_str(); }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// LoopGraph: one WHILE node, body captured into the node's child graph
// ---------------------------------------------------------------------------
void loop_graph_begin(cudaGraph_t *g, cudaGraphConditionalHandle *h, cudaGraph_t *body, cudaStream_t *cap) {
    HM_CUDA_CHECK(cudaGraphCreate(g, 0));
    HM_CUDA_CHECK(cudaGraphConditionalHandleCreate(h, *g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = *h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    HM_CUDA_CHECK(cudaGraphAddNode(&node, *g, nullptr, nullptr, 0, &np));
    *body = np.conditional.phGraph_out[0];
    HM_CUDA_CHECK(cudaStreamCreateWithFlags(cap, cudaStreamNonBlocking));
    HM_CUDA_CHECK(cudaStreamBeginCaptureToGraph(*cap, *body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
}

void loop_graph_end(LoopGraph &L, cudaGraph_t g, cudaGraph_t body, cudaStream_t cap, bool ok, long long launches) {
    cudaGraph_t captured = body;
    const cudaError_t ec = cudaStreamEndCapture(cap, &captured);
    cudaStreamDestroy(cap);
    if (!ok || ec != cudaSuccess) {
        cudaGraphDestroy(g);
        if (ok) fail(HM_ECUDA, "graph capture of the Arnoldi loop failed: %s", cudaGetErrorString(ec));
        return;
    }
    // the captured launches run on replay; they are counted there
    g_launches.fetch_sub(launches, std::memory_order_relaxed);
    L.body_launches = launches;
    const cudaError_t ei = cudaGraphInstantiate(&L.exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        L.exec = nullptr;
        fail(HM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    }
}

LoopGraph::~LoopGraph() {
    if (exec) cudaGraphExecDestroy(exec);
}

void LoopGraph::launch(cudaStream_t s) const { HM_CUDA_CHECK(cudaGraphLaunch(exec, s)); }

void LoopGraph::count(long long iterations) const {
    g_launches.fetch_add(body_launches * iterations, std::memory_order_relaxed);
}

// ----------------------------------------------------------------------------
// kernel timing trace
// ----------------------------------------------------------------------------
namespace {
struct TraceRec {
    const char *name;
    cudaEvent_t a, b;
};
std::mutex g_trace_mu;
std::atomic<bool> g_trace_on{false};
std::vector<TraceRec> g_trace_recs;
std::vector<cudaEvent_t> g_trace_pool;

cudaEvent_t trace_event() {  // caller holds g_trace_mu
    if (!g_trace_pool.empty()) {
        cudaEvent_t e = g_trace_pool.back();
        g_trace_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    HM_CUDA_CHECK(cudaEventCreate(&e));
    return e;
}
}  // namespace

Trace::Trace(const char *name, cudaStream_t stream) : s(stream) {
    if (!g_trace_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HM_CUDA_CHECK(cudaStreamIsCapturing(stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    TraceRec r{name, trace_event(), trace_event()};
    HM_CUDA_CHECK(cudaEventRecord(r.a, stream));
    slot = (int)g_trace_recs.size();
    g_trace_recs.push_back(r);
}

Trace::~Trace() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (slot < (int)g_trace_recs.size()) cudaEventRecord(g_trace_recs[slot].b, s);
}

void trace_enable(bool on) {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (on) {
        for (auto &r : g_trace_recs) {
            HM_CUDA_CHECK(cudaEventSynchronize(r.b));
            g_trace_pool.push_back(r.a);
            g_trace_pool.push_back(r.b);
        }
        g_trace_recs.clear();
    }
    g_trace_on.store(on);
}

std::vector<TraceTotal> trace_read() {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    std::vector<TraceTotal> out;
    for (auto &r : g_trace_recs) {
        HM_CUDA_CHECK(cudaEventSynchronize(r.b));
        float ms = 0.0f;
        HM_CUDA_CHECK(cudaEventElapsedTime(&ms, r.a, r.b));
        size_t k = 0;
        while (k < out.size() && out[k].name != r.name) ++k;
        if (k == out.size()) out.push_back(TraceTotal{r.name, 0, 0.0});
        out[k].launches += 1;
        out[k].ms += ms;
    }
    return out;
}

void fail(hm_status s, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw Failure{s, std::string(buf)};
}

// ----------------------------------------------------------------------------
// device buffers
// ----------------------------------------------------------------------------
// block cache of DBuf (see hm_internal.cuh)
constexpr size_t CACHE_MIN = size_t(1) << 20;
static std::mutex g_cache_mu;
static std::multimap<std::pair<int, size_t>, void *> g_cache;  // (device, size) -> block
static size_t g_cache_bytes = 0;

static size_t cache_cap() {
    static size_t cap = 0;
    if (!cap) {
        size_t fr = 0, tot = 0;
        cap = cudaMemGetInfo(&fr, &tot) == cudaSuccess ? tot / 4 : (size_t(8) << 30);
    }
    return cap;
}

void cache_trim() {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_cache) {
        cudaSetDevice(kv.first.first);
        cudaFree(kv.second);
    }
    cudaSetDevice(cur);
    g_cache.clear();
    g_cache_bytes = 0;
}

// ----------------------------------------------------------------------------
// injected allocation failures and the wait limit
// ----------------------------------------------------------------------------
static std::mutex g_fault_mu;
static long long g_fault_left = 0;  // allocations until the injected failure; 0 = off
static long long g_fault_seen = 0;  // allocations since the injection was armed

void set_fault_injection(long long n) {
    std::lock_guard<std::mutex> lk(g_fault_mu);
    g_fault_left = n > 0 ? n : 0;
    g_fault_seen = 0;
}

// HM_FAULT_INJECT=<n> arms the injection when the library is loaded
static const int g_fault_env = [] {
    const char *e = std::getenv("HM_FAULT_INJECT");
    if (e && *e) set_fault_injection(std::atoll(e));
    return 0;
}();

void fault_checkpoint(size_t nbytes) {
    long long k = 0;
    {
        std::lock_guard<std::mutex> lk(g_fault_mu);
        if (g_fault_left == 0) return;
        ++g_fault_seen;
        if (--g_fault_left != 0) return;
        k = g_fault_seen;
    }
    fail(HM_ENOMEM, "injected allocation failure (allocation %lld since arming, %zu bytes)", k, nbytes);
}

static std::atomic<long long> g_wait_limit{WAIT_LIMIT_DEFAULT};
long long wait_limit() { return g_wait_limit.load(); }
void set_wait_limit(long long cycles) { g_wait_limit.store(cycles >= 0 ? cycles : WAIT_LIMIT_DEFAULT); }

void DBuf::alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    fault_checkpoint(nbytes);
    HM_CUDA_CHECK(cudaGetDevice(&dev));
    if (nbytes >= CACHE_MIN) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.lower_bound({dev, nbytes});
        if (it != g_cache.end() && it->first.first == dev && it->first.second <= nbytes + nbytes / 8) {
            p = it->second;
            blk = it->first.second;
            bytes = nbytes;
            g_cache_bytes -= blk;
            g_cache.erase(it);
            return;
        }
    }
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        cache_trim();
        e = cudaMalloc(&p, nbytes);
    }
    if (e != cudaSuccess) {
        p = nullptr;
        (void)cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, "cudaMalloc(%zu bytes): %s", nbytes,
             cudaGetErrorString(e));
    }
    bytes = nbytes;
    blk = nbytes;
}

// Waits for the work queued on device `dev` (the device a block belongs to,
// which need not be the current one).  The library releases no buffer while
// one of its streams is being captured: buffers that captured work uses are
// allocated before the capture and released after it.
static bool sync_device(int dev) {
    int cur = dev;
    if (cudaGetDevice(&cur) != cudaSuccess) return false;
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return false;
    const bool ok = cudaDeviceSynchronize() == cudaSuccess;
    if (cur != dev) cudaSetDevice(cur);
    return ok;
}

void DBuf::release() {
    if (p) {
        bool cached = false;
        if (blk >= CACHE_MIN && sync_device(dev)) {
            std::lock_guard<std::mutex> lk(g_cache_mu);
            if (g_cache_bytes + blk <= cache_cap()) {
                g_cache.insert({{dev, blk}, p});
                g_cache_bytes += blk;
                cached = true;
            }
        }
        if (!cached) cudaFree(p);
    }
    p = nullptr;
    bytes = blk = 0;
}

int num_sms() {
    int dev = 0, sms = 0;
    HM_CUDA_CHECK(cudaGetDevice(&dev));
    HM_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
}

// ----------------------------------------------------------------------------
// quadrature constants
// ----------------------------------------------------------------------------
QuadParams make_quad(int ss_order) {
    QuadParams q{};
    // Degree-5 symmetric 7-point rule on the triangle (Radon; Stroud T2:5-1):
    // centroid with weight 9/40 and two 3-point orbits (a, a, 1-2a) with
    // a = (6 -+ sqrt 15)/21 and weights (155 -+ sqrt 15)/1200.
    const double r15 = std::sqrt(15.0);
    const double a[2] = {(6.0 - r15) / 21.0, (6.0 + r15) / 21.0};
    const double wa[2] = {(155.0 - r15) / 1200.0, (155.0 + r15) / 1200.0};
    q.bary[0][0] = q.bary[0][1] = q.bary[0][2] = 1.0 / 3.0;
    q.w[0] = 9.0 / 40.0;
    for (int o = 0; o < 2; ++o) {
        const double b = 1.0 - 2.0 * a[o];
        const double pts[3][3] = {{a[o], a[o], b}, {a[o], b, a[o]}, {b, a[o], a[o]}};
        for (int k = 0; k < 3; ++k) {
            for (int c = 0; c < 3; ++c) q.bary[1 + 3 * o + k][c] = pts[k][c];
            q.w[1 + 3 * o + k] = wa[o];
        }
    }
    for (int k = 0; k < NQ; ++k) {
        q.w_h[k] = (float)q.w[k];
        q.w_l[k] = (float)(q.w[k] - (double)q.w_h[k]);
    }
    // Gauss-Legendre on [-1, 1]: roots of P_n by Newton's method started from
    // cos(pi (k + 3/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2); then
    // mapped to [0, 1].
    const int n = ss_order;
    q.ss_n = n;
    for (int k = 0; k < n; ++k) {
        double x = std::cos(M_PI * (k + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int l = 2; l <= n; ++l) {
                double p2 = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 0) ? 1.0 : (n == 1 ? x : p1);
            double pnm1 = (n == 1) ? 1.0 : p0;
            dp = n * (x * pn - pnm1) / (x * x - 1.0);
            double dx = pn / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) {
                // one more evaluation of dp at the converged root
                p0 = 1.0;
                p1 = x;
                for (int l = 2; l <= n; ++l) {
                    double p2 = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / l;
                    p0 = p1;
                    p1 = p2;
                }
                pn = (n == 1) ? x : p1;
                pnm1 = (n == 1) ? 1.0 : p0;
                dp = n * (x * pn - pnm1) / (x * x - 1.0);
                break;
            }
        }
        double w = 2.0 / ((1.0 - x * x) * dp * dp);
        q.gx[k] = 0.5 * (x + 1.0);
        q.gw[k] = 0.5 * w;
    }
    return q;
}

// ----------------------------------------------------------------------------
// exclusive scan of int64 (three passes: tile sums, scan of sums, tile scan)
// ----------------------------------------------------------------------------
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *s_warp, int64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < nw ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    int64_t before = warp > 0 ? s_warp[warp - 1] : 0;
    if (total) *total = s_warp[nw - 1];
    return before + x - v;
}

__global__ void scan_tile_sums(const int64_t *in, int64_t n, int64_t *sums) {
    __shared__ int64_t s_warp[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t acc = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += in[i];
    }
    int64_t tot;
    block_exclusive_scan(acc, s_warp, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums_single(int64_t *sums, int64_t nb, int64_t *total) {
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = i < nb ? sums[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan(v, s_warp, &tot);
        int64_t carry = s_carry;
        if (i < nb) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = s_carry;
}

__global__ void scan_tiles(const int64_t *in, int64_t *out, int64_t n, const int64_t *sums) {
    __shared__ int64_t s_warp[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t acc = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        acc += v[k];
    }
    int64_t ex = block_exclusive_scan(acc, s_warp, nullptr) + sums[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
}

int64_t exclusive_scan_i64(const int64_t *d_in, int64_t *d_out, int64_t n, cudaStream_t s) {
    if (n <= 0) return 0;
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    DBuf sums;
    sums.alloc(sizeof(int64_t) * (nb + 1));
    int64_t *d_sums = sums.as<int64_t>();
    scan_tile_sums<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(d_in, n, d_sums);
    HM_LAUNCH_CHECK();
    scan_sums_single<<<1, 1024, 0, s>>>(d_sums, nb, d_sums + nb);
    HM_LAUNCH_CHECK();
    scan_tiles<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(d_in, d_out, n, d_sums);
    HM_LAUNCH_CHECK();
    return read_scalar(d_sums + nb, s);
}

// ----------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits.  Per pass: per-tile digit counts,
// scan of the digit-major count matrix, then an in-order scatter in which
// every tile ranks its keys stably (warp match + per-warp digit counts).
// ----------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void radix_hist(const uint64_t *keys, int64_t n, int shift, int64_t *counts, int64_t ntiles) {
    __shared__ int s_cnt[256];
    s_cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int k = 0; k < RS_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&s_cnt[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = s_cnt[threadIdx.x];
}

__global__ void radix_scatter(const uint64_t *kin, const int32_t *vin, uint64_t *kout, int32_t *vout, int64_t n,
                              int shift, const int64_t *offs, int64_t ntiles) {
    __shared__ int64_t s_base[256];
    __shared__ int s_cnt[RS_WARPS][256];
    __shared__ int s_run[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    s_run[tid] = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        for (int w = 0; w < RS_WARPS; ++w) s_cnt[w][tid] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)r * RS_THREADS + tid;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0ull;
        int32_t val = valid ? vin[i] : 0;
        unsigned d = valid ? (unsigned)((key >> shift) & 255u) : 256u + (unsigned)lane;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) s_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int run = s_run[tid];
            for (int w = 0; w < RS_WARPS; ++w) {
                int c = s_cnt[w][tid];
                s_cnt[w][tid] = run;
                run += c;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        if (valid) {
            int64_t dst = s_base[d] + s_cnt[warp][d] + rank;
            kout[dst] = key;
            vout[dst] = val;
        }
        __syncthreads();
    }
}

void radix_sort_u64(uint64_t *d_keys, int32_t *d_vals, uint64_t *d_tmp_keys, int32_t *d_tmp_vals, int64_t n,
                    int key_bits, cudaStream_t s) {
    if (n <= 1) return;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    DBuf counts;
    counts.alloc(sizeof(int64_t) * 256 * ntiles);
    int passes = (key_bits + 7) / 8;
    uint64_t *ka = d_keys, *kb = d_tmp_keys;
    int32_t *va = d_vals, *vb = d_tmp_vals;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        radix_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, n, shift, counts.as<int64_t>(), ntiles);
        HM_LAUNCH_CHECK();
        exclusive_scan_i64(counts.as<int64_t>(), counts.as<int64_t>(), 256 * ntiles, s);
        radix_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, counts.as<int64_t>(), ntiles);
        HM_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != d_keys) {
        HM_CUDA_CHECK(cudaMemcpyAsync(d_keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        HM_CUDA_CHECK(cudaMemcpyAsync(d_vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
}

__global__ void gather_i32_kernel(const int32_t *src, const int32_t *idx, int32_t *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

void gather_i32(const int32_t *d_src, const int32_t *d_idx, int32_t *d_dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    gather_i32_kernel<<<blocks, 256, 0, s>>>(d_src, d_idx, d_dst, n);
    HM_LAUNCH_CHECK();
}

// ----------------------------------------------------------------------------
// TMA tensor maps
// ----------------------------------------------------------------------------
typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(p);
    });
    if (!fn) fail(HM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    return fn;
}

// 2-D FP64 tensor [dim1][dim0] (dim0 innermost), box [box1][box0], zero fill
// out of bounds.  dim0 * 8 bytes must be a multiple of 16.
void make_tensor_map_2d_f64(CUtensorMap *map, const double *base, uint64_t dim0, uint64_t dim1, uint32_t box0,
                            uint32_t box1) {
    if ((dim0 * sizeof(double)) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || box0 > 256 ||
        box1 > 256 || (box0 * sizeof(double)) % 16 != 0)
        fail(HM_EINTERNAL, "tensor map geometry violates TMA alignment rules");
    cuuint64_t dims[2] = {dim0, dim1};
    cuuint64_t strides[1] = {dim0 * sizeof(double)};
    cuuint32_t box[2] = {box0, box1};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = get_encode()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(base), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(HM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
}

void make_tensor_map_2d_f32(CUtensorMap *map, const float *base, uint64_t dim0, uint64_t dim1, uint32_t box0,
                            uint32_t box1) {
    if ((dim0 * sizeof(float)) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || box0 > 256 ||
        box1 > 256 || (box0 * sizeof(float)) % 16 != 0)
        fail(HM_EINTERNAL, "tensor map geometry violates TMA alignment rules");
    cuuint64_t dims[2] = {dim0, dim1};
    cuuint64_t strides[1] = {dim0 * sizeof(float)};
    cuuint32_t box[2] = {box0, box1};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = get_encode()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(HM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
}

}  // namespace hm
