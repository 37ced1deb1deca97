// hm_internal.cuh -- internal declarations of the GB300 H-matrix BEM library.
//
// Device data layout (Morton order throughout; "Npad" = n rounded up to 8):
//   panel table PT : double [PT_ROWS][Npad]; row q (0..6) = x of the 7 quadrature
//                    points, rows 7..13 = y, rows 14..20 = z, row 21 = |T|,
//                    rows 22..24 = the three vertex indices (exact as doubles).
//                    Component-major so that one 2-D TMA box stages a whole
//                    cluster of panels, and consecutive panels are consecutive
//                    doubles in shared memory (conflict-free per-lane loads).
//   dense near field: one row-major panel per leaf row cluster rho, of
//                    |rho| x Kd_rho, Kd_rho = sum of the widths of the
//                    non-admissible leaves in rho's block row (concatenated in
//                    column order) rounded up to a multiple of 8, so that every
//                    row starts on a 16-byte boundary in FP64, FP32 and BF16;
//                    padding columns hold 0.  Block b's entry (i, j) lives at
//                    dense_base[b] + i * dense_ld[b] + j.
//   low-rank rows:   for each rho a second row-major panel |rho| x Ku_rho that
//                    concatenates U_b(rows of rho, :) over the admissible
//                    leaves b whose rows cover rho (Ku_rho = sum of their
//                    ranks, rounded up to 8), with the index t_off[b] + l of
//                    the projection each column multiplies.
//   W factors:       per admissible leaf, W_b row-major (n_b x k_b) at w_off[b]
//                    in a compact arena; the block is U_b W_b^T.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/hm.h"

namespace hm {

constexpr int NQ = 7;          // points of the triangle rule
constexpr int PT_ROWS = 25;    // rows of the panel table
constexpr int PT_AREA = 21;
constexpr int PT_VID = 22;
constexpr int MAX_SS = 16;     // largest Gauss-Legendre order for touching pairs
constexpr int MAX_LEAF = 256;  // largest C_leaf
constexpr int MAX_KMAX = 128;  // largest ACA rank

// ----------------------------------------------------------------------------
// errors: internal code throws hm::Failure; the C ABI converts it to a status
// ----------------------------------------------------------------------------
struct Failure {
    hm_status status;
    std::string msg;
};

void set_last_error(const std::string &msg);
[[noreturn]] void fail(hm_status s, const char *fmt, ...);

#define HM_CUDA_CHECK(call)                                                                        \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            ::hm::fail(e_ == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, "%s:%d %s: %s",     \
                       __FILE__, __LINE__, #call, cudaGetErrorString(e_));                         \
    } while (0)

// Every kernel launch is followed by HM_LAUNCH_CHECK(), which also counts it.
void count_launch();
#define HM_LAUNCH_CHECK()                  \
    do {                                   \
        ::hm::count_launch();              \
        HM_CUDA_CHECK(cudaGetLastError()); \
    } while (0)

// Kernel timing trace: while enabled (hm_trace_enable), a Trace object
// records a CUDA event on the launching stream when it is made and another
// when it goes out of scope, so the launches between them are timed on the
// device; nothing is recorded while the stream is being captured.
struct Trace {
    int slot = -1;
    cudaStream_t s = nullptr;
    Trace(const char *name, cudaStream_t stream);
    ~Trace();
    Trace(const Trace &) = delete;
    Trace &operator=(const Trace &) = delete;
};
void trace_enable(bool on);
struct TraceTotal {
    std::string name;
    long long launches;
    double ms;
};
std::vector<TraceTotal> trace_read();

// ----------------------------------------------------------------------------
// device memory: RAII buffer (cudaMalloc / cudaFree behind a block cache)
//
// Unmapping device memory costs ~0.4 ms per GB on this part, and an assembly
// frees tens of GB of temporaries, so a released buffer of at least 1 MiB is
// kept in a per-device cache (after a device synchronisation, the same wait a
// cudaFree implies) and a later allocation takes the smallest cached block
// that is large enough and at most 1/8 larger.  The cache holds at most a
// quarter of the device memory; a failed cudaMalloc empties it and retries;
// hm_trim() returns it to the driver.
// ----------------------------------------------------------------------------
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;  // requested size
    size_t blk = 0;    // size of the underlying block
    int dev = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), bytes(o.bytes), blk(o.blk), dev(o.dev) {
        o.p = nullptr;
        o.bytes = o.blk = 0;
    }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            blk = o.blk;
            dev = o.dev;
            o.p = nullptr;
            o.bytes = o.blk = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t nbytes);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};
void cache_trim();  // frees every cached block

// Injected allocation failures (hm_set_fault_injection, HM_FAULT_INJECT): every
// device allocation of the library (DBuf, SBuf) passes this checkpoint first;
// the armed one throws HM_ENOMEM as a failed cudaMalloc would.
void fault_checkpoint(size_t nbytes);
void set_fault_injection(long long n);

// Limit, in SM clock cycles, of the device-side bounded waits (hm_set_wait_limit).
constexpr long long WAIT_LIMIT_DEFAULT = 4000000000LL;  // ~2 s at 2 GHz
long long wait_limit();
void set_wait_limit(long long cycles);

// Stream-ordered scratch (cudaMallocAsync / cudaFreeAsync on one stream): the
// memory is usable by work queued on that stream after the allocation and is
// returned to the pool after the work queued before the release, so a call
// that only needs temporary space does not synchronise.
struct SBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    SBuf() = default;
    SBuf(const SBuf &) = delete;
    SBuf &operator=(const SBuf &) = delete;
    ~SBuf() {
        if (p) cudaFreeAsync(p, s);
    }
    void alloc(size_t nbytes, cudaStream_t stream) {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        s = stream;
        fault_checkpoint(nbytes);
        HM_CUDA_CHECK(cudaMallocAsync(&p, nbytes ? nbytes : 16, stream));
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Reads a device value synchronously on `s`.
template <class T> T read_scalar(const T *d, cudaStream_t s) {
    T h;
    HM_CUDA_CHECK(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    HM_CUDA_CHECK(cudaStreamSynchronize(s));
    return h;
}

int num_sms();

// ----------------------------------------------------------------------------
// Device-driven loops as CUDA graphs (prims.cu).  A LoopGraph holds one
// WHILE conditional node whose body is captured once from `body` on a private
// stream; the body's last kernel decides, on the device, whether another
// iteration runs (cudaGraphSetConditional on the handle it is given).  The
// handle starts at 1 on every launch, so the body runs at least once; a body
// must clear it after a bounded number of iterations.
// ----------------------------------------------------------------------------
struct LoopCtl {       // device-side state of an Arnoldi loop
    int j;             // next step of the cycle
    int lim;           // steps allowed in this cycle
    double thr;        // stopping threshold of the residual estimate
};

struct LoopGraph {
    cudaGraphExec_t exec = nullptr;
    long long body_launches = 0;  // kernels of one iteration
    LoopGraph() = default;
    LoopGraph(const LoopGraph &) = delete;
    LoopGraph &operator=(const LoopGraph &) = delete;
    ~LoopGraph();
    template <class F> void build(F &&body);  // body(cudaStream_t, cudaGraphConditionalHandle)
    void launch(cudaStream_t s) const;
    void count(long long iterations) const;  // adds the replayed kernels to the launch count
};

void loop_graph_begin(cudaGraph_t *g, cudaGraphConditionalHandle *h, cudaGraph_t *body, cudaStream_t *cap);
void loop_graph_end(LoopGraph &L, cudaGraph_t g, cudaGraph_t body, cudaStream_t cap, bool ok, long long launches);
long long launch_count();

template <class F> void LoopGraph::build(F &&body) {
    cudaGraph_t g, bg;
    cudaGraphConditionalHandle h;
    cudaStream_t cap;
    loop_graph_begin(&g, &h, &bg, &cap);
    const long long before = launch_count();
    try {
        body(cap, h);
    } catch (...) {
        loop_graph_end(*this, g, bg, cap, false, 0);
        throw;
    }
    loop_graph_end(*this, g, bg, cap, true, launch_count() - before);
}

// ----------------------------------------------------------------------------
// quadrature data passed by value to kernels (lives in the parameter bank)
// ----------------------------------------------------------------------------
struct QuadParams {
    double bary[NQ][3];  // 7-point rule, barycentric
    double w[NQ];        // weights, sum 1
    int ss_n;            // Gauss-Legendre order on [0, 1] for touching pairs
    double gx[MAX_SS];
    double gw[MAX_SS];
    float w_h[NQ];       // the 7 weights as float pairs (w = w_h + w_l)
    float w_l[NQ];
};

// 7-point rule from its closed form; Gauss-Legendre nodes by Newton's method
// on the Legendre polynomial (three-term recurrence).
QuadParams make_quad(int ss_order);

// ----------------------------------------------------------------------------
// primitives (prims.cu)
// ----------------------------------------------------------------------------
// exclusive scan of n int64 values (in may equal out); returns the total
int64_t exclusive_scan_i64(const int64_t *d_in, int64_t *d_out, int64_t n, cudaStream_t s);
// stable ascending sort of 64-bit keys with 32-bit payloads (LSD radix);
// keys/vals are sorted in place, d_tmp_* are scratch of the same sizes
void radix_sort_u64(uint64_t *d_keys, int32_t *d_vals, uint64_t *d_tmp_keys, int32_t *d_tmp_vals, int64_t n,
                    int key_bits, cudaStream_t s);
void gather_i32(const int32_t *d_src, const int32_t *d_idx, int32_t *d_dst, int64_t n, cudaStream_t s);

// ----------------------------------------------------------------------------
// TMA tensor maps (driver entry point resolved through the runtime)
// ----------------------------------------------------------------------------
void make_tensor_map_2d_f64(CUtensorMap *map, const double *base, uint64_t dim0, uint64_t dim1, uint32_t box0,
                            uint32_t box1);
void make_tensor_map_2d_f32(CUtensorMap *map, const float *base, uint64_t dim0, uint64_t dim1, uint32_t box0,
                            uint32_t box1);

}  // namespace hm

// ----------------------------------------------------------------------------
// the opaque handles of the C ABI
// ----------------------------------------------------------------------------
constexpr uint32_t HM_TREE_MAGIC = 0x48545245u;    // "HTRE"
constexpr uint32_t HM_MATRIX_MAGIC = 0x484d4154u;  // "HMAT"

struct hm_tree {
    uint32_t magic = HM_TREE_MAGIC;
    int64_t n = 0, nv = 0, npad = 0;
    int32_t leaf = 0;
    double eta = 0.0;
    hm::DBuf V;        // [nv][3] double, copy of the caller's vertices
    hm::DBuf trim;     // [n][3] int32, triangles in Morton order
    hm::DBuf pt;       // [PT_ROWS][npad] double, panel table (Morton order)
    hm::DBuf pf;       // [PF_ROWS][npad] float, far-field panel table (see ff.cuh)
    hm::DBuf cent;     // [n][3] double, centroids in Morton order
    hm::DBuf perm;     // [n] int32, Morton position -> original index
    hm::DBuf iperm;    // [n] int32, original index -> Morton position
    // cluster tree
    int64_t n_clusters = 0;
    int32_t depth = 0;
    hm::DBuf cl_range;  // [nc][2] int32 (begin, end), breadth-first
    hm::DBuf cl_box;    // [nc][6] double (lo xyz, hi xyz)
    int64_t n_leaf = 0;
    int32_t max_leaf = 0;
    // geometries of a batched tree: panels of geometry g occupy the Morton
    // positions [geom_off[g], geom_off[g + 1]) (host copy; one geometry = [0, n))
    std::vector<int64_t> geom_off;
    hm::DBuf leaf_begin;  // [n_leaf + 1] int32, begins of the leaf clusters (ascending)
    // block tree
    int64_t n_dense = 0, n_adm = 0;
    hm::DBuf dense;       // [n_dense][4] int32, sorted by (row_begin, col_begin), rows = one leaf cluster
    hm::DBuf dense_base;  // [n_dense] int64, offset of entry (0, 0) in the near-field arena
    hm::DBuf dense_ld;    // [n_dense] int32, row stride in the arena
    hm::DBuf dense_tp;    // [n_dense] int32, leaf with swapped ranges, or -1
    int64_t dense_entries = 0;  // arena size (with row padding)
    int64_t dense_true = 0;     // sum over non-admissible leaves of |tau||sigma|
    hm::DBuf rho_off;     // [n_leaf + 1] int64, arena offset of each leaf row cluster's panel
    hm::DBuf rho_K;       // [n_leaf] int32, width of the panel
    hm::DBuf rho_colptr;  // [n_leaf + 1] int64, into colidx
    hm::DBuf colidx;      // [sum Kd] int32, Morton column of each panel column (0 for padding)
    int32_t max_dense_dim = 0;
    hm::DBuf adm;         // [n_adm][4] int32, in block-tree level order (largest first)
    hm::DBuf adm_tp;      // [n_adm] int32, leaf with swapped ranges, or -1
    int64_t adm_rows_cols = 0;
    hm::DBuf lr_rowptr;   // [n_leaf + 1] int64: admissible leaves whose rows cover each leaf cluster
    hm::DBuf lr_list;     // [..] int32 block ids (ascending per leaf cluster)
    hm::DBuf lr_colptr;   // [n_leaf + 1] int64: admissible leaves whose columns cover each leaf cluster
    hm::DBuf lr_collist;  // [..] int32 block ids (ascending per leaf cluster)
    hm::DBuf lr_bcolptr;  // [n_adm + 1] int64: first (block, column leaf cluster) pair of each block
    hm::DBuf lr_browptr;  // [n_adm + 1] int64: first (block, row leaf cluster) pair of each block
    int64_t singular_cap = 0;  // upper bound on touching pairs
    int64_t n_singular = 0;    // filled by hm_assemble
    double seconds = 0.0;
    CUtensorMap pt_map;   // TMA map of the panel table, box [PT_ROWS][box_cols]
    int32_t box_cols = 0;
    CUtensorMap pf_map;   // TMA map of the float-pair table, box [PF_ROWS][box_cols_f]
    int32_t box_cols_f = 0;  // 0: leaves too wide for one box
};

// Working vectors of one H-matrix-vector product (Morton order).
struct MatvecWork {
    double *xm;   // [n]  input
    double *ym;   // [n]  output
    double *t;    // [total_rank] projections (FP64 product)
    double *p;    // [n_partials] per-column-cluster partial projections (FP64)
    float *x32;   // [n]  input rounded to FP32 (low-precision products)
    float *t32;   // [total_rank] projections (low-precision products)
    float *p32;   // [n_partials] partial projections (low-precision products)
};

namespace hm {
// Block-column panels of one precision (the multi-RHS projection t = W^T X):
// the W factors grouped by block column cluster (one row-major panel
// |sigma| x K_sigma per cluster sigma, the blocks with that column cluster
// side by side), the t index of every panel column (-1 = padding) and the
// work items (panel, first column, rows, partial slot) and reductions.
struct BcpSet {
    DBuf data, off, K, rows, col0, tidx, tiles, red;
    int64_t ngroups = 0, ntiles = 0, nred = 0, nslots = 0;
    int dtype = -1;  // hm_dtype of data, -1 = not built
};
// Row panels of one part of the factors: per leaf row cluster a row-major
// panel |rho| x K_rho, and the t index of each of its columns.
struct TailPanels {
    DBuf data, off, K, colptr, tidx;
    int64_t entries = 0;
};
}  // namespace hm

struct hm_matrix {
    uint32_t magic = HM_MATRIX_MAGIC;
    const hm_tree *tree = nullptr;
    hm_assemble_params params{};
    hm::DBuf dense;     // near-field row panels, double
    hm::DBuf dense32;   // optional FP32 copy
    hm::DBuf mv_order;  // [4][n_leaf] int32: leaf clusters by decreasing panel work
                        // (row / column kernel, forward; row / column kernel, transposed)
    hm::DBuf rank;      // [n_adm] int32
    hm::DBuf t_off;     // [n_adm] int64, prefix sum of ranks
    int64_t total_rank = 0;
    int64_t lr_entries = 0;  // sum_b k_b (m_b + n_b)
    // U_b rows, grouped by leaf row cluster
    hm::DBuf up;        // low-rank row panels, double
    hm::DBuf up32;      // optional FP32 copy
    hm::DBuf upbf;      // optional BF16 copy
    hm::DBuf up_off;    // [n_leaf + 1] int64, panel offsets
    hm::DBuf up_K;      // [n_leaf] int32, padded panel widths
    hm::DBuf up_colptr; // [n_leaf + 1] int64, into tidx
    hm::DBuf tidx;      // [sum Ku] int32, projection index of each panel column (0 for padding)
    hm::DBuf up_koff;   // [lr_list size] int32, first panel column of each (rho, block) pair
    int64_t up_entries = 0;
    // W_b rows, grouped by leaf column cluster kappa: panel |kappa| x Kw
    hm::DBuf wp;        // low-rank column panels, double
    hm::DBuf wp32;      // optional FP32 copy
    hm::DBuf wpbf;      // optional BF16 copy
    hm::DBuf wp_off;    // [n_leaf + 1] int64, panel offsets
    hm::DBuf wp_K;      // [n_leaf] int32, padded panel widths
    hm::DBuf wp_colptr; // [n_leaf + 1] int64, into the partial-projection vector
    hm::DBuf wp_koff;   // [lr_collist size] int32, first panel column of each (kappa, block) pair
    hm::DBuf pofs;      // [sum over blocks of column leaf clusters] int64: partial offsets per block
    hm::DBuf tsum_b0;   // [ceil(total_rank / 32)] int32: block holding t entry 32 c
    // transposed product (built on first use): the near field of H^T in the
    // layout of the row panels (and its FP32 rounding), the partial offsets
    // of the projections through the U panels, and the t index of every W
    // panel column
    hm::DBuf dense_t, dense32_t, pofs_t, tidx_t;
    int64_t n_partials_t = 0;
    bool trans_ready = false;
    // multi-RHS projection (built on first use for a precision)
    hm::BcpSet bcp;     // the W factors of the copy (with BF16 tails: the leading terms)
    hm::BcpSet bcp16;   // with BF16 tails: the trailing terms, BF16
    hm::DBuf mrhs_err;  // [1] int: a bounded wait of the tensor-memory row pass gave up (0 = none)
    // FP32 factors with BF16 tails (params.factor_tail_bits > 0): per
    // admissible block the number of its leading ACA terms kept in FP32 (the
    // trailing ones, each below 2^-bits of the block's largest term, are kept
    // in BF16 for the 16-RHS product), and the row panels of the two parts
    // (built with the FP32 copy), in the layout of the master's row panels
    hm::DBuf rank32;    // [n_adm] int32
    hm::DBuf rank16;    // [n_adm] int32: k_b - k32_b
    hm::TailPanels ut32, ut16;
    int64_t wp_entries = 0;
    int64_t n_partials = 0;  // length of the partial-projection vector
    // block-Jacobi preconditioner: inverse of each leaf cluster's diagonal block
    // block-Jacobi preconditioner (built on the first preconditioned solve):
    // inverses of the near-field diagonal blocks of runs of leaf clusters,
    // column-major per block
    hm::DBuf bj;        // [sum m_b^2] double
    hm::DBuf bj32;      // its FP32 rounding (preconditioner of the inner solves)
    hm::DBuf bj_off;    // [n_bj + 1] int64
    hm::DBuf bj_begin;  // [n_bj + 1] int32: first row of each block
    hm::DBuf bj_leaf;   // [n_bj + 1] int32: first leaf cluster of each block
    int64_t n_bj = 0;
    int bj_mmax = 0;    // rows of the largest block
    hm_matrix_info info{};
};
