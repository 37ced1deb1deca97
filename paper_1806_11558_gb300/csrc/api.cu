// api.cu -- the extern "C" entry points declared in include/hm.h.
//
// Every entry point validates its arguments on the host before queueing any
// device work, converts internal failures (hm::Failure) into an hm_status and
// records a message for hm_last_error().  A bounded device-side wait that gives
// up is reported through a device error word and becomes HM_ETIMEOUT.
#include <chrono>
#include <cmath>
#include <memory>

#include "hm_internal.cuh"

namespace hm {
const char *last_error_cstr();
long long launch_count();
hm_tree *build_tree_impl(const double *d_V, int64_t nv, const int32_t *d_T, int64_t n, const hm_tree_params &prm,
                         cudaStream_t s);
void assemble_nearfield(const hm_tree *tr, hm_matrix *A, const QuadParams &qp, cudaStream_t s, int *d_err,
                        double *sec_regular, double *sec_singular);
void assemble_aca(const hm_tree *tr, hm_matrix *A, const QuadParams &qp, cudaStream_t s, double *sec);
void make_low_copies(hm_matrix *A, cudaStream_t s);
void matvec_morton(const hm_matrix *A, hm_dtype prec, const MatvecWork &w, cudaStream_t s);
int64_t matvec_work_doubles(const hm_matrix *A);
MatvecWork matvec_work_at(const hm_matrix *A, double *base);
void build_lr_desc(hm_matrix *A, cudaStream_t s);
void permute_to_morton(const hm_tree *tr, const double *x, double *xm, cudaStream_t s);
void permute_from_morton(const hm_tree *tr, const double *ym, double alpha, double beta, double *y, cudaStream_t s);
void load_vector_impl(const hm_tree *tr, const double *src, int nsrc, double *f, cudaStream_t s);
hm_status solve_impl(const hm_matrix *A, const double *b, double *x, const hm_solve_params &p, cudaStream_t s,
                     hm_solve_info *info);
void matvec_noalloc(const hm_matrix *A, int32_t nrhs, hm_dtype prec, const double *x, double *y, double alpha,
                    double beta, cudaStream_t s);
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
        *out = build_tree_impl(d_vertices, n_vertices, d_tris, n_tris, *params, (cudaStream_t)stream);
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
        assemble_nearfield(tree, A.get(), qp, s, err.as<int>(), &sr, &ss);
        assemble_aca(tree, A.get(), qp, s, &sa);
        build_lr_desc(A.get(), s);
        make_low_copies(A.get(), s);
        HM_CUDA_CHECK(cudaStreamSynchronize(s));
        const int e = read_scalar(err.as<int>(), s);
        if (e == 2) fail(HM_ETIMEOUT, "a panel staging wait timed out");
        if (e) fail(HM_EINTERNAL, "device error code %d during assembly", e);
        hm_matrix_info &I = A->info;
        I.dense_entries = tree->dense_entries;
        I.lr_entries = A->lr_entries;
        I.s_nearfield = sr;
        I.s_singular = ss;
        I.s_aca = sa;
        I.bytes_f64 = (int64_t)(A->dense.bytes + A->uw.bytes);
        I.bytes_low = (int64_t)(A->dense32.bytes + A->uw32.bytes + A->uwbf.bytes);
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

hm_status hm_matvec(const hm_matrix *A, int32_t trans, int32_t nrhs, hm_dtype prec, const double *d_x, double *d_y,
                    double alpha, double beta, hm_stream_t stream) {
    return guard([&] {
        if (!is_matrix(A)) fail(HM_EINVAL, "not a matrix handle");
        if (!d_x || !d_y) fail(HM_EINVAL, "NULL argument");
        if (nrhs < 1) fail(HM_EINVAL, "nrhs must be >= 1");
        if (trans != 0 && trans != 1) fail(HM_EINVAL, "trans must be 0 or 1");
        if (trans == 1) fail(HM_EINVAL, "the transposed product is not available in this build");
        if (prec == HM_F32 && !A->uw32.p) fail(HM_EINVAL, "FP32 copies were not assembled");
        if (prec == HM_BF16 && !A->uwbf.p) fail(HM_EINVAL, "BF16 factors were not assembled");
        if (prec < HM_F64 || prec > HM_BF16) fail(HM_EINVAL, "bad precision");
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t n = A->tree->n;
        DBuf work;
        work.alloc(sizeof(double) * matvec_work_doubles(A));
        const MatvecWork w = matvec_work_at(A, work.as<double>());
        for (int r = 0; r < nrhs; ++r) {
            permute_to_morton(A->tree, d_x + (int64_t)r * n, w.xm, s);
            matvec_morton(A, prec, w, s);
            permute_from_morton(A->tree, w.ym, alpha, beta, d_y + (int64_t)r * n, s);
        }
        HM_CUDA_CHECK(cudaStreamSynchronize(s));
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
        if (prec == HM_F32 && !A->uw32.p) fail(HM_EINVAL, "FP32 copies were not assembled");
        if (prec == HM_BF16 && !A->uwbf.p) fail(HM_EINVAL, "BF16 factors were not assembled");
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
        if (trans == 1) fail(HM_EINVAL, "the transposed solve is not available in this build");
        if (params->restart < 1 || params->restart > 128) fail(HM_EINVAL, "restart must be in [1, 128]");
        if (params->max_iter < 1) fail(HM_EINVAL, "max_iter must be >= 1");
        if (!(params->rel_tol > 0.0)) fail(HM_EINVAL, "rel_tol must be > 0");
        if (params->refine) {
            if (params->max_refine < 1) fail(HM_EINVAL, "max_refine must be >= 1");
            if (!(params->inner_tol > 0.0)) fail(HM_EINVAL, "inner_tol must be > 0");
            if (params->inner_dtype == HM_F32 && !A->uw32.p) fail(HM_EINVAL, "FP32 copies were not assembled");
            if (params->inner_dtype == HM_BF16 && !A->uwbf.p) fail(HM_EINVAL, "BF16 factors were not assembled");
            if (params->inner_dtype < HM_F64 || params->inner_dtype > HM_BF16) fail(HM_EINVAL, "bad inner_dtype");
        }
        const int64_t n = A->tree->n;
        for (int r = 0; r < nrhs; ++r) {
            hm_status st = solve_impl(A, d_b + (int64_t)r * n, d_x + (int64_t)r * n, *params, (cudaStream_t)stream, info);
            if (st != HM_OK) {
                result = st;
                set_last_error("GMRES reached max_iter before rel_tol");
            }
        }
    });
    return g != HM_OK ? g : result;
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
        info->n_dense = tree->n_dense;
        info->n_adm = tree->n_adm;
        info->dense_entries = tree->dense_entries;
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
        *n_dense_vals = tr->dense_entries;
        *n_lr_vals = A->lr_entries;
        if (!h_dense && !h_uw) return;
        if (!h_dense || !h_dense_off || !h_rank || !h_uw || !h_u_off || !h_w_off) fail(HM_EINVAL, "NULL buffer");
        const int64_t nd = tr->n_dense, na = tr->n_adm;
        std::vector<int32_t> den(4 * nd), adm(4 * na), ld(nd), rank(na);
        std::vector<int64_t> base(nd), uwo(na);
        std::vector<double> arena(tr->dense_entries);
        if (nd) {
            HM_CUDA_CHECK(cudaMemcpy(den.data(), tr->dense.p, sizeof(int32_t) * 4 * nd, cudaMemcpyDeviceToHost));
            HM_CUDA_CHECK(cudaMemcpy(base.data(), tr->dense_base.p, sizeof(int64_t) * nd, cudaMemcpyDeviceToHost));
            HM_CUDA_CHECK(cudaMemcpy(ld.data(), tr->dense_ld.p, sizeof(int32_t) * nd, cudaMemcpyDeviceToHost));
            HM_CUDA_CHECK(cudaMemcpy(arena.data(), A->dense.p, sizeof(double) * tr->dense_entries,
                                     cudaMemcpyDeviceToHost));
        }
        int64_t o = 0;
        for (int64_t b = 0; b < nd; ++b) {
            const int m = den[4 * b + 1] - den[4 * b], n = den[4 * b + 3] - den[4 * b + 2];
            h_dense_off[b] = o;
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < n; ++j) h_dense[o + (int64_t)i * n + j] = arena[base[b] + (int64_t)i * ld[b] + j];
            o += (int64_t)m * n;
        }
        std::vector<double> fac(std::max<int64_t>(A->lr_entries, 1));
        if (na) {
            HM_CUDA_CHECK(cudaMemcpy(adm.data(), tr->adm.p, sizeof(int32_t) * 4 * na, cudaMemcpyDeviceToHost));
            HM_CUDA_CHECK(cudaMemcpy(rank.data(), A->rank.p, sizeof(int32_t) * na, cudaMemcpyDeviceToHost));
            HM_CUDA_CHECK(cudaMemcpy(uwo.data(), A->uw_off.p, sizeof(int64_t) * na, cudaMemcpyDeviceToHost));
            HM_CUDA_CHECK(cudaMemcpy(fac.data(), A->uw.p, sizeof(double) * A->lr_entries, cudaMemcpyDeviceToHost));
        }
        // U_b as stored (column-major); W_b stored row-major, exported column-major
        for (int64_t b = 0; b < na; ++b) {
            const int m = adm[4 * b + 1] - adm[4 * b], n = adm[4 * b + 3] - adm[4 * b + 2], k = rank[b];
            h_rank[b] = k;
            h_u_off[b] = uwo[b];
            h_w_off[b] = uwo[b] + (int64_t)m * k;
            for (int64_t e = 0; e < (int64_t)m * k; ++e) h_uw[uwo[b] + e] = fac[uwo[b] + e];
            for (int j = 0; j < n; ++j)
                for (int l = 0; l < k; ++l)
                    h_uw[h_w_off[b] + (int64_t)l * n + j] = fac[h_w_off[b] + (int64_t)j * k + l];
        }
    });
}

}  // extern "C"
