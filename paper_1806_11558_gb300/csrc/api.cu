// api.cu -- the extern "C" entry points declared in include/hm.h.
//
// Every entry point validates its arguments on the host before queueing any
// device work, converts internal failures (hm::Failure) into an hm_status and
// records a message for hm_last_error().  A bounded device-side wait that gives
// up is reported through a device error word and becomes HM_ETIMEOUT.
#include <chrono>
#include <cmath>
#include <memory>

#include <cstring>

#include "hm_internal.cuh"

namespace hm {
const char *last_error_cstr();
long long launch_count();
hm_tree *build_tree_impl(const double *d_V, int64_t nv, const int32_t *d_T, int64_t n, const hm_tree_params &prm,
                         const std::vector<int64_t> &goff, cudaStream_t s);
void load_vector_geom_impl(const hm_tree *tr, const double *src, int nsrc, double *f, cudaStream_t s);
void assemble_nearfield(const hm_tree *tr, hm_matrix *A, const QuadParams &qp, cudaStream_t s, int *d_err,
                        double *sec_regular, double *sec_singular, bool fp64);
void assemble_aca(const hm_tree *tr, hm_matrix *A, const QuadParams &qp, cudaStream_t s, double *sec, DBuf &uw,
                  DBuf &uw_off);
void build_lr_panels(hm_matrix *A, const DBuf &uw, const DBuf &uw_off, cudaStream_t s);
void ensure_f32_copies(const hm_matrix *A, cudaStream_t s);
void ensure_bf16_copies(const hm_matrix *A, cudaStream_t s);
void make_low_copies(hm_matrix *A, cudaStream_t s);
void split_terms(hm_matrix *A, const DBuf &uw, const DBuf &uw_off, cudaStream_t s);
void matvec_morton(const hm_matrix *A, hm_dtype prec, const MatvecWork &w, cudaStream_t s, bool trans);
void build_transposed(const hm_matrix *A, cudaStream_t s);
int64_t matvec_work_doubles(const hm_matrix *A);
MatvecWork matvec_work_at(const hm_matrix *A, double *base);
void permute_to_morton(const hm_tree *tr, const double *x, double *xm, cudaStream_t s);
void permute_from_morton(const hm_tree *tr, const double *ym, double alpha, double beta, double *y, cudaStream_t s);
void load_vector_impl(const hm_tree *tr, const double *src, int nsrc, double *f, cudaStream_t s);
hm_status solve_impl(const hm_matrix *A, const double *b, double *x, const hm_solve_params &p, cudaStream_t s,
                     hm_solve_info *info, bool trans);
void get_block(const hm_matrix *A, int dense, int64_t b, double *out, cudaStream_t s);
hm_status solve_batched(const hm_matrix *A, int nrhs, const double *b_orig, double *x_orig, const hm_solve_params &p,
                        cudaStream_t s, hm_solve_info *info);
void matvec_mrhs(const hm_matrix *A, hm_dtype prec, int nrhs, const double *x, double *y, double alpha, double beta,
                 cudaStream_t s);
void potential_impl(const hm_tree *tr, const double *pts, int64_t K, int trans, const double *in, double *out,
                    cudaStream_t s);
void matvec_noalloc(const hm_matrix *A, int32_t nrhs, hm_dtype prec, const double *x, double *y, double alpha,
                    double beta, cudaStream_t s);
double measure_fma_peak(hm_dtype kind, cudaStream_t s);
int mrhs_error(const hm_matrix *A, cudaStream_t s);
void matvec_df(const hm_matrix *A, int nrhs, const double *x, double *y, double alpha, double beta, cudaStream_t s);
void div_diag(const double *a, const double *d, int64_t n, int nrhs, double *out, cudaStream_t s);
void mul_diag(const double *a, const double *d, int64_t n, int nrhs, double *out, cudaStream_t s);
void axpby_diag(const double *v, const double *d, int64_t n, int nrhs, double alpha, double beta, double *y,
                cudaStream_t s);
}  // namespace hm

using namespace hm;

template <class F> static hm_status guard(F &&f) {
    try {
        set_last_error("");
        f();
        return HM_OK;
    } catch (const Failure &e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return HM_ENOMEM;
    } catch (...) {
        set_last_error("unexpected internal exception");
        return HM_EINTERNAL;
    }
}

static bool is_tree(const void *p) { return p && static_cast<const hm_tree *>(p)->magic == HM_TREE_MAGIC; }
static bool is_matrix(const void *p) { return p && static_cast<const hm_matrix *>(p)->magic == HM_MATRIX_MAGIC; }

static void check_matvec_args(const hm_matrix *A, int32_t trans, int32_t nrhs, hm_dtype prec, const double *d_x,
                              const double *d_y) {
    if (!is_matrix(A)) fail(HM_EINVAL, "not a matrix handle");
    if (!d_x || !d_y) fail(HM_EINVAL, "NULL argument");
    if (nrhs < 1) fail(HM_EINVAL, "nrhs must be >= 1");
    if (trans != 0 && trans != 1) fail(HM_EINVAL, "trans must be 0 or 1");
    if (prec < HM_F64 || prec > HM_BF16) fail(HM_EINVAL, "bad precision");
    if (prec == HM_F32 && !A->up32.p) fail(HM_EINVAL, "FP32 copies were not assembled");
    if (prec == HM_BF16 && !A->upbf.p) fail(HM_EINVAL, "BF16 factors were not assembled");
}

// y = alpha op(H) x + beta y, [nrhs][n] in original order, one right-hand side at a time
static void matvec_orig(const hm_matrix *A, int32_t trans, int32_t nrhs, hm_dtype prec, const double *d_x,
                        double *d_y, double alpha, double beta, cudaStream_t s) {
    const int64_t n = A->tree->n;
    SBuf work;
    work.alloc(sizeof(double) * matvec_work_doubles(A), s);
    const MatvecWork w = matvec_work_at(A, work.as<double>());
    if (trans) build_transposed(A, s);
    for (int r = 0; r < nrhs; ++r) {
        permute_to_morton(A->tree, d_x + (int64_t)r * n, w.xm, s);
        matvec_morton(A, prec, w, s, trans == 1);
        permute_from_morton(A->tree, w.ym, alpha, beta, d_y + (int64_t)r * n, s);
    }
}

extern "C" {

const char *hm_last_error(void) { return last_error_cstr(); }

int64_t hm_kernel_launches(void) { return (int64_t)launch_count(); }

hm_status hm_build_tree(const double *d_vertices, int64_t n_vertices, const int32_t *d_tris, int64_t n_tris,
                        const hm_tree_params *params, hm_stream_t stream, hm_tree **out) {
    if (out) *out = nullptr;
    return guard([&] {
        if (!out || !d_vertices || !d_tris || !params) fail(HM_EINVAL, "NULL argument");
        if (n_tris < 1 || n_tris > (1LL << 28)) fail(HM_EINVAL, "n_tris must be in [1, 2^28]");
        if (n_vertices < 3 || n_vertices > (1LL << 30)) fail(HM_EINVAL, "n_vertices must be in [3, 2^30]");
        if (!(params->eta >= 0.0) || !std::isfinite(params->eta)) fail(HM_EINVAL, "eta must be finite and >= 0");
        if (params->leaf_size < 1 || params->leaf_size > 254) fail(HM_EINVAL, "leaf_size must be in [1, 254]");
        *out = build_tree_impl(d_vertices, n_vertices, d_tris, n_tris, *params, {}, (cudaStream_t)stream);
    });
}

hm_status hm_build_forest(const double *d_vertices, int64_t n_vertices, const int32_t *d_tris, int64_t n_tris,
                          const int64_t *h_tri_offsets, int32_t n_geom, const hm_tree_params *params,
                          hm_stream_t stream, hm_tree **out) {
    if (out) *out = nullptr;
    return guard([&] {
        if (!out || !d_vertices || !d_tris || !params || !h_tri_offsets) fail(HM_EINVAL, "NULL argument");
        if (n_tris < 1 || n_tris > (1LL << 28)) fail(HM_EINVAL, "n_tris must be in [1, 2^28]");
        if (n_vertices < 3 || n_vertices > (1LL << 30)) fail(HM_EINVAL, "n_vertices must be in [3, 2^30]");
        if (n_geom < 1 || n_geom > 65536) fail(HM_EINVAL, "n_geom must be in [1, 65536]");
        if (!(params->eta >= 0.0) || !std::isfinite(params->eta)) fail(HM_EINVAL, "eta must be finite and >= 0");
        if (params->leaf_size < 1 || params->leaf_size > 254) fail(HM_EINVAL, "leaf_size must be in [1, 254]");
        std::vector<int64_t> goff(h_tri_offsets, h_tri_offsets + n_geom + 1);
        if (goff[0] != 0 || goff[n_geom] != n_tris) fail(HM_EINVAL, "tri_offsets must start at 0 and end at n_tris");
        for (int g = 0; g < n_geom; ++g)
            if (goff[g + 1] <= goff[g]) fail(HM_EINVAL, "geometry %d has no triangle", g);
        *out = build_tree_impl(d_vertices, n_vertices, d_tris, n_tris, *params, goff, (cudaStream_t)stream);
    });
}

hm_status hm_load_vector_geom(const hm_tree *tree, const double *d_sources, int32_t n_per_geom, double *d_f,
                              hm_stream_t stream) {
    return guard([&] {
        if (!is_tree(tree)) fail(HM_EINVAL, "not a tree handle");
        if (!d_sources || !d_f) fail(HM_EINVAL, "NULL argument");
        if (n_per_geom < 1) fail(HM_EINVAL, "n_per_geom must be >= 1");
        load_vector_geom_impl(tree, d_sources, n_per_geom, d_f, (cudaStream_t)stream);
    });
}

hm_status hm_assemble(const hm_tree *tree, const hm_assemble_params *params, hm_stream_t stream, hm_matrix **out) {
    if (out) *out = nullptr;
    return guard([&] {
        if (!out || !params) fail(HM_EINVAL, "NULL argument");
        if (!is_tree(tree)) fail(HM_EINVAL, "not a tree handle");
        if (!(params->aca_eps > 0.0) || !std::isfinite(params->aca_eps)) fail(HM_EINVAL, "aca_eps must be > 0");
        if (params->aca_kmax < 1 || params->aca_kmax > MAX_KMAX) fail(HM_EINVAL, "aca_kmax must be in [1, 128]");
        if (params->ss_order < 1 || params->ss_order > MAX_SS) fail(HM_EINVAL, "ss_order must be in [1, 16]");
        if (params->factor_dtype < HM_F64 || params->factor_dtype > HM_BF16) fail(HM_EINVAL, "bad factor_dtype");
        if (params->dense_dtype != HM_F64 && params->dense_dtype != HM_F32) fail(HM_EINVAL, "bad dense_dtype");
        if (params->nearfield_fp64 != 0 && params->nearfield_fp64 != 1) fail(HM_EINVAL, "nearfield_fp64 must be 0 or 1");
        if (params->mrhs_tcgen05 != 0 && params->mrhs_tcgen05 != 1) fail(HM_EINVAL, "mrhs_tcgen05 must be 0 or 1");
        if (params->factor_tail_bits != 0 && (params->factor_tail_bits < 8 || params->factor_tail_bits > 24))
            fail(HM_EINVAL, "factor_tail_bits must be 0 or in [8, 24]");
        cudaStream_t s = (cudaStream_t)stream;
        const auto t0 = std::chrono::steady_clock::now();
        std::unique_ptr<hm_matrix> A(new hm_matrix());
        A->tree = tree;
        A->params = *params;
        const QuadParams qp = make_quad(params->ss_order);
        DBuf err;
        err.alloc(sizeof(int));
        HM_CUDA_CHECK(cudaMemsetAsync(err.p, 0, sizeof(int), s));
        double sr = 0, ss = 0, sa = 0;
        assemble_nearfield(tree, A.get(), qp, s, err.as<int>(), &sr, &ss, params->nearfield_fp64 != 0);
        {
            DBuf uw, uw_off;
            assemble_aca(tree, A.get(), qp, s, &sa, uw, uw_off);
            build_lr_panels(A.get(), uw, uw_off, s);
            if (params->factor_tail_bits > 0) split_terms(A.get(), uw, uw_off, s);
            HM_CUDA_CHECK(cudaStreamSynchronize(s));
        }
        make_low_copies(A.get(), s);
        HM_CUDA_CHECK(cudaStreamSynchronize(s));
        const int e = read_scalar(err.as<int>(), s);
        if (e == 2) fail(HM_ETIMEOUT, "a panel staging wait timed out");
        if (e) fail(HM_EINTERNAL, "device error code %d during assembly", e);
        hm_matrix_info &I = A->info;  // mean / max rank, kmax hits and ACA entries are set by the ACA
        I.dense_entries = tree->dense_true;
        I.lr_entries = A->lr_entries;
        I.s_nearfield = sr;
        I.s_singular = ss;
        I.s_aca = sa;
        I.bytes_f64 = (int64_t)(A->dense.bytes + A->up.bytes + A->wp.bytes);
        I.bytes_low = (int64_t)(A->dense32.bytes + A->up32.bytes + A->upbf.bytes + A->wp32.bytes + A->wpbf.bytes +
                                A->ut32.data.bytes + A->ut16.data.bytes);
        I.s_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        *out = A.release();
    });
}

hm_status hm_load_vector(const hm_tree *tree, const double *d_sources, int32_t n_sources, double *d_f,
                         hm_stream_t stream) {
    return guard([&] {
        if (!is_tree(tree)) fail(HM_EINVAL, "not a tree handle");
        if (!d_sources || !d_f) fail(HM_EINVAL, "NULL argument");
        if (n_sources < 1) fail(HM_EINVAL, "n_sources must be >= 1");
        load_vector_impl(tree, d_sources, n_sources, d_f, (cudaStream_t)stream);
    });
}

hm_status hm_potential(const hm_tree *tree, const double *d_points, int64_t n_points, int32_t trans,
                       const double *d_in, double *d_out, hm_stream_t stream) {
    return guard([&] {
        if (!is_tree(tree)) fail(HM_EINVAL, "not a tree handle");
        if (n_points < 0) fail(HM_EINVAL, "n_points must be >= 0");
        if (trans != 0 && trans != 1) fail(HM_EINVAL, "trans must be 0 or 1");
        const bool reads = trans ? n_points > 0 : true, writes = trans ? true : n_points > 0;
        if ((n_points > 0 && !d_points) || (reads && !d_in) || (writes && !d_out)) fail(HM_EINVAL, "NULL argument");
        potential_impl(tree, d_points, n_points, trans, d_in, d_out, (cudaStream_t)stream);
    });
}

hm_status hm_matvec(const hm_matrix *A, int32_t trans, int32_t nrhs, hm_dtype prec, const double *d_x, double *d_y,
                    double alpha, double beta, hm_stream_t stream) {
    return guard([&] {
        check_matvec_args(A, trans, nrhs, prec, d_x, d_y);
        matvec_orig(A, trans, nrhs, prec, d_x, d_y, alpha, beta, (cudaStream_t)stream);
    });
}

hm_status hm_matvec_scaled(const hm_matrix *A, int32_t trans, int32_t nrhs, hm_dtype prec, const double *d_left,
                           const double *d_right, const double *d_x, double *d_y, double alpha, double beta,
                           hm_stream_t stream) {
    return guard([&] {
        check_matvec_args(A, trans, nrhs, prec, d_x, d_y);
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t n = A->tree->n;
        SBuf xs, ys;
        const double *xin = d_x;
        if (d_right) {
            xs.alloc(sizeof(double) * n * nrhs, s);
            mul_diag(d_x, d_right, n, nrhs, xs.as<double>(), s);
            xin = xs.as<double>();
        }
        ys.alloc(sizeof(double) * n * nrhs, s);
        matvec_orig(A, trans, nrhs, prec, xin, ys.as<double>(), 1.0, 0.0, s);
        axpby_diag(ys.as<double>(), d_left, n, nrhs, alpha, beta, d_y, s);
    });
}

hm_status hm_matvec_block(const hm_matrix *A, int32_t nrhs, hm_dtype prec, const double *d_x, double *d_y,
                          double alpha, double beta, hm_stream_t stream) {
    return guard([&] {
        if (!is_matrix(A)) fail(HM_EINVAL, "not a matrix handle");
        if (!d_x || !d_y) fail(HM_EINVAL, "NULL argument");
        if (nrhs < 1) fail(HM_EINVAL, "nrhs must be >= 1");
        if (prec != HM_F64 && prec != HM_F32 && prec != HM_BF16) fail(HM_EINVAL, "unknown precision %d", (int)prec);
        if (prec == HM_F64) {  // the FP64 master in double-float arithmetic (mrhs_df.cu)
            matvec_df(A, nrhs, d_x, d_y, alpha, beta, (cudaStream_t)stream);
            return;
        }
        if (!A->dense32.p || (prec == HM_F32 ? !A->up32.p : !A->upbf.p))
            fail(HM_EINVAL, "the low-precision copies for this precision were not assembled");
        matvec_mrhs(A, prec, nrhs, d_x, d_y, alpha, beta, (cudaStream_t)stream);
        // the tcgen05 row pass reports a bounded wait that gave up (the form compared, not the default)
        if (A->params.mrhs_tcgen05 && mrhs_error(A, (cudaStream_t)stream))
            fail(HM_ETIMEOUT, "a bounded wait of the tensor-memory row pass gave up");
    });
}

hm_status hm_matvec_noalloc(const hm_matrix *A, int32_t trans, int32_t nrhs, hm_dtype prec, const double *d_x,
                            double *d_y, double alpha, double beta, hm_stream_t stream) {
    return guard([&] {
        if (!is_matrix(A)) fail(HM_EINVAL, "not a matrix handle");
        if (!d_x || !d_y) fail(HM_EINVAL, "NULL argument");
        if (nrhs < 1) fail(HM_EINVAL, "nrhs must be >= 1");
        if (trans != 0) fail(HM_EINVAL, "only trans = 0 is available");
        if (prec < HM_F64 || prec > HM_BF16) fail(HM_EINVAL, "bad precision");
        if (prec == HM_F32 && !A->up32.p) fail(HM_EINVAL, "FP32 copies were not assembled");
        if (prec == HM_BF16 && !A->upbf.p) fail(HM_EINVAL, "BF16 factors were not assembled");
        matvec_noalloc(A, nrhs, prec, d_x, d_y, alpha, beta, (cudaStream_t)stream);
    });
}

hm_status hm_solve(const hm_matrix *A, int32_t trans, int32_t nrhs, const double *d_b, double *d_x,
                   const hm_solve_params *params, hm_stream_t stream, hm_solve_info *info) {
    hm_status result = HM_OK;
    hm_status g = guard([&] {
        if (!is_matrix(A)) fail(HM_EINVAL, "not a matrix handle");
        if (!d_b || !d_x || !params) fail(HM_EINVAL, "NULL argument");
        if (nrhs < 1) fail(HM_EINVAL, "nrhs must be >= 1");
        if (trans != 0 && trans != 1) fail(HM_EINVAL, "trans must be 0 or 1");
        if (params->restart < 1 || params->restart > 128) fail(HM_EINVAL, "restart must be in [1, 128]");
        if (params->precond != 0 && params->precond != 1) fail(HM_EINVAL, "precond must be 0 or 1");
        if (params->max_iter < 1) fail(HM_EINVAL, "max_iter must be >= 1");
        if (!(params->rel_tol > 0.0)) fail(HM_EINVAL, "rel_tol must be > 0");
        if (params->refine) {
            if (params->max_refine < 1) fail(HM_EINVAL, "max_refine must be >= 1");
            if (!(params->inner_tol > 0.0)) fail(HM_EINVAL, "inner_tol must be > 0");
            if (params->inner_dtype == HM_F32 && !A->up32.p) fail(HM_EINVAL, "FP32 copies were not assembled");
            if (params->inner_dtype == HM_BF16 && !A->upbf.p) fail(HM_EINVAL, "BF16 factors were not assembled");
            if (params->inner_dtype < HM_F64 || params->inner_dtype > HM_BF16) fail(HM_EINVAL, "bad inner_dtype");
        }
        if (params->batched != 0 && params->batched != 1) fail(HM_EINVAL, "batched must be 0 or 1");
        if (params->use_graph != 0 && params->use_graph != 1) fail(HM_EINVAL, "use_graph must be 0 or 1");
        if (std::isnan(params->stall_ratio)) fail(HM_EINVAL, "stall_ratio is NaN");
        if (params->resid_df != 0 && params->resid_df != 1) fail(HM_EINVAL, "resid_df must be 0 or 1");
        if (params->batched && trans) fail(HM_EINVAL, "the batched solve is for trans = 0");
        if (params->batched && params->refine && params->inner_dtype != HM_F64 && !A->dense32.p)
            fail(HM_EINVAL, "the FP32 near-field copy was not assembled");
        if (params->batched) {
            const hm_status st = solve_batched(A, nrhs, d_b, d_x, *params, (cudaStream_t)stream, info);
            if (st != HM_OK) {
                result = st;
                set_last_error("GMRES reached max_iter (or max_refine) before rel_tol");
            }
            return;
        }
        const int64_t n = A->tree->n;
        if (trans) build_transposed(A, (cudaStream_t)stream);
        for (int r = 0; r < nrhs; ++r) {
            hm_status st = solve_impl(A, d_b + (int64_t)r * n, d_x + (int64_t)r * n, *params, (cudaStream_t)stream, info,
                                      trans == 1);
            if (st != HM_OK) {
                result = st;
                set_last_error("GMRES reached max_iter before rel_tol");
            }
        }
    });
    return g != HM_OK ? g : result;
}

hm_status hm_solve_scaled(const hm_matrix *A, int32_t trans, int32_t nrhs, const double *d_c, const double *d_b,
                          double *d_x, const hm_solve_params *params, hm_stream_t stream, hm_solve_info *info) {
    hm_status g = guard([&] {
        if (!is_matrix(A)) fail(HM_EINVAL, "not a matrix handle");
        if (!d_c || !d_b || !d_x || !params) fail(HM_EINVAL, "NULL argument");
        if (nrhs < 1) fail(HM_EINVAL, "nrhs must be >= 1");
        if (trans != 0 && trans != 1) fail(HM_EINVAL, "trans must be 0 or 1");
    });
    if (g != HM_OK) return g;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->tree->n;
    if (trans == 0) {
        // H diag(c) x = b  <=>  H y = b, x = y / c
        const hm_status st = hm_solve(A, 0, nrhs, d_b, d_x, params, stream, info);
        if (st != HM_OK && st != HM_ENOCONV) return st;
        const std::string msg = last_error_cstr();
        g = guard([&] { div_diag(d_x, d_c, n, nrhs, d_x, s); });
        if (g != HM_OK) return g;
        set_last_error(msg);
        return st;
    }
    // (H diag(c))^T x = diag(c) H^T x = b  <=>  H^T x = b / c
    SBuf bc;
    g = guard([&] {
        bc.alloc(sizeof(double) * n * nrhs, s);
        div_diag(d_b, d_c, n, nrhs, bc.as<double>(), s);
    });
    if (g != HM_OK) return g;
    return hm_solve(A, 1, nrhs, bc.as<double>(), d_x, params, stream, info);
}

hm_status hm_matrix_add_copy(const hm_matrix *A, hm_dtype dtype, hm_stream_t stream) {
    return guard([&] {
        if (!is_matrix(A)) fail(HM_EINVAL, "not a matrix handle");
        if (dtype != HM_F32 && dtype != HM_BF16) fail(HM_EINVAL, "dtype must be HM_F32 or HM_BF16");
        if (dtype == HM_F32)
            ensure_f32_copies(A, (cudaStream_t)stream);
        else
            ensure_bf16_copies(A, (cudaStream_t)stream);
    });
}

void hm_trim(void) {
    cudaDeviceSynchronize();
    cache_trim();
}

void hm_free(void *handle) {
    if (is_matrix(handle)) {
        hm_matrix *A = static_cast<hm_matrix *>(handle);
        A->magic = 0;
        delete A;
    } else if (is_tree(handle)) {
        hm_tree *t = static_cast<hm_tree *>(handle);
        t->magic = 0;
        delete t;
    }
}

hm_status hm_tree_get_info(const hm_tree *tree, hm_tree_info *info) {
    return guard([&] {
        if (!is_tree(tree) || !info) fail(HM_EINVAL, "bad argument");
        info->n = tree->n;
        info->n_clusters = tree->n_clusters;
        info->depth = tree->depth;
        info->max_leaf = tree->max_leaf;
        info->n_geom = tree->geom_off.size() > 1 ? (int32_t)tree->geom_off.size() - 1 : 1;
        info->n_dense = tree->n_dense;
        info->n_adm = tree->n_adm;
        info->dense_entries = tree->dense_true;
        info->adm_rows_cols = tree->adm_rows_cols;
        info->n_singular = tree->n_singular;
        info->seconds = tree->seconds;
    });
}

hm_status hm_tree_get_perm(const hm_tree *tree, int32_t *d_perm) {
    return guard([&] {
        if (!is_tree(tree) || !d_perm) fail(HM_EINVAL, "bad argument");
        HM_CUDA_CHECK(cudaMemcpy(d_perm, tree->perm.p, sizeof(int32_t) * tree->n, cudaMemcpyDeviceToDevice));
    });
}

hm_status hm_tree_get_leaves(const hm_tree *tree, int32_t dense, int32_t *d_out, int64_t capacity, int64_t *count) {
    return guard([&] {
        if (!is_tree(tree) || !count) fail(HM_EINVAL, "bad argument");
        const int64_t n = dense ? tree->n_dense : tree->n_adm;
        *count = n;
        if (d_out && capacity >= n && n > 0)
            HM_CUDA_CHECK(cudaMemcpy(d_out, dense ? tree->dense.p : tree->adm.p, sizeof(int32_t) * 4 * n,
                                     cudaMemcpyDeviceToDevice));
    });
}

hm_status hm_set_wait_limit(int64_t cycles) {
    set_wait_limit((long long)cycles);
    return HM_OK;
}

hm_status hm_set_fault_injection(int64_t n) {
    set_fault_injection((long long)n);
    return HM_OK;
}

hm_status hm_measure_fma_peak(hm_dtype kind, double *tflops, hm_stream_t stream) {
    return guard([&] {
        if (!tflops) fail(HM_EINVAL, "NULL argument");
        if (kind != HM_F64 && kind != HM_F32) fail(HM_EINVAL, "kind must be HM_F64 or HM_F32");
        *tflops = measure_fma_peak(kind, (cudaStream_t)stream);
    });
}

hm_status hm_trace_enable(int32_t on) {
    return guard([&] { trace_enable(on != 0); });
}

hm_status hm_trace_read(hm_trace_entry *out, int32_t capacity, int32_t *count) {
    return guard([&] {
        if (!count) fail(HM_EINVAL, "NULL count");
        const std::vector<TraceTotal> t = trace_read();
        *count = (int32_t)t.size();
        for (int32_t k = 0; out && k < capacity && k < (int32_t)t.size(); ++k) {
            std::memset(out[k].name, 0, sizeof(out[k].name));
            std::strncpy(out[k].name, t[k].name.c_str(), sizeof(out[k].name) - 1);
            out[k].launches = t[k].launches;
            out[k].ms = t[k].ms;
        }
    });
}

hm_status hm_matrix_get_block(const hm_matrix *A, int32_t dense, int64_t index, double *d_out, hm_stream_t stream) {
    return guard([&] {
        if (!is_matrix(A) || !d_out) fail(HM_EINVAL, "bad argument");
        get_block(A, dense != 0, index, d_out, (cudaStream_t)stream);
    });
}

hm_status hm_matrix_get_info(const hm_matrix *A, hm_matrix_info *info) {
    return guard([&] {
        if (!is_matrix(A) || !info) fail(HM_EINVAL, "bad argument");
        *info = A->info;
    });
}

hm_status hm_matrix_export(const hm_matrix *A, double *h_dense, int64_t *h_dense_off, int32_t *h_rank, double *h_uw,
                           int64_t *h_u_off, int64_t *h_w_off, int64_t *n_dense_vals, int64_t *n_lr_vals) {
    return guard([&] {
        if (!is_matrix(A) || !n_dense_vals || !n_lr_vals) fail(HM_EINVAL, "bad argument");
        const hm_tree *tr = A->tree;
        *n_dense_vals = tr->dense_true;
        *n_lr_vals = A->lr_entries;
        if (!h_dense && !h_uw) return;
        if (!h_dense || !h_dense_off || !h_rank || !h_uw || !h_u_off || !h_w_off) fail(HM_EINVAL, "NULL buffer");
        const int64_t nd = tr->n_dense, na = tr->n_adm, nl = tr->n_leaf;
        auto get = [](void *dst, const DBuf &src, size_t bytes) {
            if (bytes) HM_CUDA_CHECK(cudaMemcpy(dst, src.p, bytes, cudaMemcpyDeviceToHost));
        };
        // dense leaves, row-major per block
        std::vector<int32_t> den(4 * nd), ld(nd);
        std::vector<int64_t> base(nd);
        std::vector<double> arena(tr->dense_entries);
        get(den.data(), tr->dense, sizeof(int32_t) * 4 * nd);
        get(base.data(), tr->dense_base, sizeof(int64_t) * nd);
        get(ld.data(), tr->dense_ld, sizeof(int32_t) * nd);
        get(arena.data(), A->dense, sizeof(double) * tr->dense_entries);
        int64_t o = 0;
        for (int64_t b = 0; b < nd; ++b) {
            const int m = den[4 * b + 1] - den[4 * b], n = den[4 * b + 3] - den[4 * b + 2];
            h_dense_off[b] = o;
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < n; ++j) h_dense[o + (int64_t)i * n + j] = arena[base[b] + (int64_t)i * ld[b] + j];
            o += (int64_t)m * n;
        }
        if (na == 0) return;
        // low-rank factors: U_b gathered back from the row panels, W_b from the
        // column panels (column-major in the export)
        std::vector<int32_t> adm(4 * na), rank(na), leaf_begin(nl + 1), up_K(nl), wp_K(nl), koff, lr_list, wkoff,
            lr_collist;
        std::vector<int64_t> lr_rowptr(nl + 1), up_off(nl + 1), lr_colptr(nl + 1), wp_off(nl + 1);
        get(adm.data(), tr->adm, sizeof(int32_t) * 4 * na);
        get(rank.data(), A->rank, sizeof(int32_t) * na);
        get(leaf_begin.data(), tr->leaf_begin, sizeof(int32_t) * (nl + 1));
        get(lr_rowptr.data(), tr->lr_rowptr, sizeof(int64_t) * (nl + 1));
        get(lr_colptr.data(), tr->lr_colptr, sizeof(int64_t) * (nl + 1));
        get(up_off.data(), A->up_off, sizeof(int64_t) * (nl + 1));
        get(wp_off.data(), A->wp_off, sizeof(int64_t) * (nl + 1));
        get(up_K.data(), A->up_K, sizeof(int32_t) * nl);
        get(wp_K.data(), A->wp_K, sizeof(int32_t) * nl);
        const int64_t np = lr_rowptr[nl], npc = lr_colptr[nl];
        koff.resize(np);
        lr_list.resize(np);
        wkoff.resize(npc);
        lr_collist.resize(npc);
        get(koff.data(), A->up_koff, sizeof(int32_t) * np);
        get(lr_list.data(), tr->lr_list, sizeof(int32_t) * np);
        get(wkoff.data(), A->wp_koff, sizeof(int32_t) * npc);
        get(lr_collist.data(), tr->lr_collist, sizeof(int32_t) * npc);
        std::vector<double> up(A->up_entries), wp(A->wp_entries);
        get(up.data(), A->up, sizeof(double) * A->up_entries);
        get(wp.data(), A->wp, sizeof(double) * A->wp_entries);
        o = 0;
        for (int64_t b = 0; b < na; ++b) {
            const int m = adm[4 * b + 1] - adm[4 * b], n = adm[4 * b + 3] - adm[4 * b + 2], k = rank[b];
            h_rank[b] = k;
            h_u_off[b] = o;
            h_w_off[b] = o + (int64_t)m * k;
            o += (int64_t)(m + n) * k;
        }
        for (int64_t c = 0; c < nl; ++c) {
            const int32_t c0 = leaf_begin[c], mc = leaf_begin[c + 1] - c0;
            for (int64_t q = lr_colptr[c]; q < lr_colptr[c + 1]; ++q) {
                const int32_t b = lr_collist[q];
                const int n = adm[4 * b + 3] - adm[4 * b + 2], k = rank[b], off = c0 - adm[4 * b + 2];
                for (int j = 0; j < mc; ++j)
                    for (int l = 0; l < k; ++l)
                        h_uw[h_w_off[b] + (int64_t)l * n + off + j] = wp[wp_off[c] + (int64_t)j * wp_K[c] + wkoff[q] + l];
            }
        }
        for (int64_t r = 0; r < nl; ++r) {
            const int32_t r0 = leaf_begin[r], mr = leaf_begin[r + 1] - r0;
            for (int64_t q = lr_rowptr[r]; q < lr_rowptr[r + 1]; ++q) {
                const int32_t b = lr_list[q];
                const int m = adm[4 * b + 1] - adm[4 * b], k = rank[b], off = r0 - adm[4 * b];
                for (int i = 0; i < mr; ++i)
                    for (int l = 0; l < k; ++l)
                        h_uw[h_u_off[b] + (int64_t)l * m + off + i] = up[up_off[r] + (int64_t)i * up_K[r] + koff[q] + l];
            }
        }
    });
}

}  // extern "C"
