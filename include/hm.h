/*
 * hm.h -- C ABI of the GB300 H-matrix boundary-element library.
 *
 * Method: Harbrecht & Zaspel, "A scalable H-matrix approach for the solution
 * of boundary integral equations on multi-GPU clusters" (arXiv 1806.11558):
 * a Galerkin discretisation of the single-layer Laplace operator
 * (Sec. 2.1 Example 2.1, Sec. 2.2 Eq. 4) with piecewise-constant elements on
 * flat triangles, approximated by an H-matrix (Sec. 2.3: Morton-ordered
 * cluster tree, Algorithm 1 block tree under Eq. 5, dense near field,
 * adaptive cross approximation of admissible blocks), applied in an
 * H-matrix-vector product and solved by a Krylov method (Sec. 4.1).
 *
 * Conventions shared by every call
 *  - Pointers named d_* are CUDA device pointers owned by the caller; the
 *    library never frees them.  Handles (hm_tree, hm_matrix) are owned by the
 *    library until hm_free.  A matrix keeps a reference to its tree: free the
 *    matrix before the tree.
 *  - User vectors are in the caller's original panel order (the index maps
 *    idx_1 = idx_2 = "the index of the panel" of Sec. 3.2); the Morton
 *    permutation is applied internally.
 *  - Calls are ordered on `stream` (NULL = the legacy default stream).  Calls
 *    that report host-side results (counts, info structs) synchronise the
 *    stream before returning.
 *  - Every call returns an hm_status.  On failure no output handle is
 *    created (*out is set to NULL) and hm_last_error() describes the cause.
 *    Argument errors are detected before any computation is queued (the
 *    vertex-index range check of hm_build_tree is a small device kernel that
 *    runs before anything else).
 *  - Kernels never trap: every bounded wait that gives up makes the call
 *    return HM_ETIMEOUT with the device context left usable.
 */
#ifndef HM_H
#define HM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Symbols of the C ABI are the only ones the shared library exports. */
#if defined(__GNUC__)
#define HM_API __attribute__((visibility("default")))
#else
#define HM_API
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *hm_stream_t;

typedef enum {
    HM_OK = 0,
    HM_EINVAL = 1,     /* invalid argument (sizes, NULL pointers, ranges)            */
    HM_ENOMEM = 2,     /* device or host allocation failed                           */
    HM_ECUDA = 3,      /* a CUDA runtime / driver call failed                        */
    HM_ENOCONV = 4,    /* the solver reached its iteration limit; best x is returned */
    HM_ETIMEOUT = 5,   /* a bounded device-side wait gave up                         */
    HM_EINTERNAL = 6   /* an internal consistency check failed                       */
} hm_status;

typedef enum { HM_F64 = 0, HM_F32 = 1, HM_BF16 = 2 } hm_dtype;

typedef struct hm_tree hm_tree;     /* opaque, library-owned */
typedef struct hm_matrix hm_matrix; /* opaque, library-owned */

/* Cluster / block tree parameters (Sec. 2.3).
 *  eta        : admissibility parameter of Eq. 5, eta >= 0.
 *  leaf_size  : C_leaf of condition (C3), 1 <= leaf_size <= 254. */
typedef struct {
    double eta;
    int32_t leaf_size;
} hm_tree_params;

/* Assembly parameters.
 *  aca_eps      : relative ACA stopping tolerance, > 0.
 *  aca_kmax     : largest ACA rank per block, 1 <= aca_kmax <= 128.
 *  ss_order     : Gauss-Legendre order of the regularised touching-pair
 *                 integrals, 1 <= ss_order <= 16.
 *  factor_dtype : HM_F64 (FP64 only), or HM_F32 / HM_BF16 to also keep a
 *                 low-precision copy of the low-rank factors.
 *  dense_dtype  : HM_F64 (FP64 only) or HM_F32 to also keep an FP32 copy of
 *                 the dense near field.
 *  nearfield_fp64 : 0 (default) = the regular near-field entries (dense
 *                 leaves, panels not touching) and the regularised integrals
 *                 of pairs sharing a vertex or an edge in double-float
 *                 arithmetic on the FP32 units (about 48 significant bits,
 *                 ~1e-14 relative), like the ACA entries; 1 = in FP64
 *                 arithmetic.  Identical panels are always FP64.  Regular
 *                 entries of leaves wider than 250 panels always use FP64.
 *  mrhs_tcgen05 : 0 (default) = the row pass of the 16-right-hand-side
 *                 product (hm_matvec_block, batched inner solves) on
 *                 mma.sync; 1 = on the fifth-generation tensor cores
 *                 (tcgen05.mma, accumulators in tensor memory).  Both give
 *                 the product to the same ~2^-16 accuracy; on a GB300 the
 *                 tcgen05 form measured about 2x slower on the level-8
 *                 sphere, so it is kept for comparison, not as the default.
 *                 Its waits are bounded: one that gives up makes the
 *                 batched solve, or hm_matvec_block (which then
 *                 synchronises its stream), return HM_ETIMEOUT.
 *  factor_tail_bits : 0 (default), or 8 ... 24: with factor_dtype = HM_F32
 *                 (or a later FP32 copy), the 16-right-hand-side product
 *                 keeps in BF16 the trailing ACA terms of every block: the
 *                 terms after the last one whose size ||u_l|| ||w_l|| is at
 *                 least 2^-factor_tail_bits of the block's largest term
 *                 (Sec. 2.3: the terms of an ACA fall roughly geometrically
 *                 to the tolerance).  Each such term's BF16 rounding is
 *                 below 2^-(9 + factor_tail_bits) of the block's largest
 *                 term, against ~2^-17 of every term from the product's
 *                 BF16-pair rounding of FP32 factors; the bytes of those
 *                 columns halve.  The single-right-hand-side FP32 product
 *                 and every FP64 product are unchanged.
 *  The FP64 master copy is always kept. */
typedef struct {
    double aca_eps;
    int32_t aca_kmax;
    int32_t ss_order;
    hm_dtype factor_dtype;
    hm_dtype dense_dtype;
    int32_t nearfield_fp64;
    int32_t mrhs_tcgen05;
    int32_t factor_tail_bits;
} hm_assemble_params;

/* Solver parameters.
 *  restart    : GMRES restart length m (GMRES(m)), 1 <= restart <= 128.
 *  max_iter   : total Arnoldi steps allowed (over all restarts / refinements).
 *  rel_tol    : stop when ||b - H x|| <= rel_tol ||b|| (FP64 residual).
 *  refine     : 0 = plain FP64 GMRES on the FP64 H-matrix;
 *               1 = iterative refinement: inner GMRES on the inner_dtype
 *                   operator (FP64 Krylov vectors, Hessenberg and Givens),
 *                   outer residual in FP64.
 *  max_refine : largest number of refinement steps (refine = 1).
 *  inner_tol  : relative tolerance of each inner solve (refine = 1).
 *  inner_dtype: HM_F32 or HM_BF16 (factors of that type, dense FP32).
 *  precond    : 0 = none (the paper's unpreconditioned Krylov solve);
 *               1 = right block-Jacobi preconditioning with the inverses of
 *                   the near-field diagonal blocks of runs of consecutive
 *                   leaf clusters of at most 200 rows (one leaf when leaves
 *                   are larger), computed on the first such solve and kept
 *                   with the matrix: inverted in FP32 (blocks of at most 232
 *                   rows; FP64 beyond), applied in FP64 by FP64 solves and
 *                   in FP32 by the inner solves.  The preconditioner only
 *                   changes the Krylov basis: the residual and the stopping
 *                   test are those of the unpreconditioned FP64 system. */
typedef struct {
    int32_t restart;
    int32_t max_iter;
    double rel_tol;
    int32_t refine;
    int32_t max_refine;
    double inner_tol;
    hm_dtype inner_dtype;
    int32_t precond;
    int32_t batched;  /* 1 = solve the nrhs systems together (trans = 0): every
                         system runs its own GMRES, in lockstep, and each
                         Arnoldi step applies H to all of them at once — on the
                         FP32 / BF16 copies through the tensor-core product of
                         hm_matvec_block (16 right-hand sides per pass), on the
                         FP64 master one column after the other.  info reports
                         the lockstep step count and the largest relative
                         residual.  0 = one system after the other. */
    int32_t use_graph; /* 1 = run the Arnoldi steps of every GMRES cycle as one
                          CUDA graph (a WHILE conditional node over one step,
                          the stop decided on the device); the host waits
                          once per cycle instead of once per step.  Same
                          kernels and arithmetic, so the same iterates as 0.
                          The graph is built on the first cycle of the call
                          (one per precision used). */
    double stall_ratio; /* refine = 1: an outer step whose FP64 residual is
                           above stall_ratio times the previous one has not
                           contracted (the inner operator is too inexact for
                           the conditioning, kappa u >~ 1), and the inner
                           precision is raised for the remaining steps:
                           HM_BF16 -> HM_F32 (FP32 copies of the factors and
                           the near field are made from the FP64 master and
                           kept with the matrix when the assembly did not keep
                           them); HM_F32 -> HM_F64.  <= 0 selects 0.5; NaN is
                           HM_EINVAL. */
    int32_t resid_df;   /* refine = 1 and batched = 1: 1 = the outer residuals
                           b - H x of all systems by the 16-right-hand-side
                           product of the FP64 master in double-float
                           arithmetic (hm_matvec_block with HM_F64: each stored
                           entry read once per 16 systems, the arithmetic on
                           the FP32 pipe; ~1e-14 of |H||x| instead of ~1e-16),
                           and the stopping test on them; 0 = one FP64 product
                           per system.  Other values: HM_EINVAL. */
} hm_solve_params;

typedef struct {
    int32_t status;       /* hm_status of the solve                               */
    int32_t iters;        /* Arnoldi steps taken (inner steps when refining)       */
    int32_t restarts;     /* GMRES cycles                                          */
    int32_t refine_steps; /* outer refinement steps (0 when refine = 0)            */
    double rel_resid;     /* final ||b - H x|| / ||b|| with the FP64 operator       */
    double seconds;       /* wall time of the call                                 */
    int32_t inner_dtype;  /* precision of the last inner solve (refine = 1; it is
                             above the requested one after a stall, see
                             stall_ratio); HM_F64 when refine = 0             */
    double kappa_est;     /* sigma_max / sigma_min of the first GMRES cycle's
                             Hessenberg matrix (of the first inner solve when
                             refining): a lower estimate of the condition
                             number of op(H) (of op(H) M^-1 with precond = 1);
                             0 for batched solves                            */
} hm_solve_info;

typedef struct {
    int64_t n;              /* panels = unknowns                                  */
    int64_t n_clusters;     /* clusters of the cluster tree                       */
    int32_t depth;          /* depth of the cluster tree                          */
    int32_t max_leaf;       /* largest leaf cluster                               */
    int64_t n_dense;        /* non-admissible leaves of the block tree            */
    int64_t n_adm;          /* admissible leaves                                  */
    int64_t dense_entries;  /* sum of |tau||sigma| over non-admissible leaves     */
    int64_t adm_rows_cols;  /* sum of |tau| + |sigma| over admissible leaves      */
    int64_t n_singular;     /* Sauter-Schwab evaluations of the last assembly:
                               touching pairs (shared vertex, edge or panel),
                               a common-vertex pair of a symmetric block
                               counted once                                    */
    double seconds;         /* wall time of hm_build_tree                         */
    int32_t n_geom;         /* geometries (1 unless built by hm_build_forest)     */
} hm_tree_info;

typedef struct {
    int64_t dense_entries;  /* stored FP64 near-field entries                     */
    int64_t lr_entries;     /* stored FP64 factor entries, sum k_b (|tau|+|sigma|) */
    int32_t max_rank;
    int32_t kmax_hit;       /* admissible blocks that stopped at aca_kmax         */
    double mean_rank;
    double s_nearfield;     /* device seconds: regular near-field kernel          */
    double s_singular;      /* device seconds: touching-pair kernel               */
    double s_aca;           /* device seconds: batched ACA kernel                 */
    double s_total;         /* wall seconds of hm_assemble                        */
    int64_t bytes_f64;      /* device bytes of the FP64 matrix data               */
    int64_t bytes_low;      /* device bytes of the low-precision copies           */
    int64_t aca_entries;    /* entries the ACA evaluated, sum k_b (|tau|+|sigma|)
                               over the blocks it approximated (the transposed
                               partner of an approximated block reuses its
                               factors, the matrix being symmetric)            */
    int64_t u_entries;      /* stored entries of the U factors, sum k_b |tau|     */
    int32_t aca_small_sum;  /* ACA worker split chosen by the autotuner: blocks
                               with m + n up to this (and both dims <= 256) run
                               on one warp, larger ones on a whole CTA        */
    int32_t aca_threads;    /* ACA launch chosen by the autotuner: threads per CTA
                               (64, 128 or 256) ...                               */
    int32_t aca_ctas_per_sm; /* ... and CTAs per SM of the persistent launch     */
    int64_t factor_tail_terms; /* ACA terms (over all admissible blocks, a
                               mirrored block counting its partner's) that
                               the 16-RHS product keeps in BF16
                               (factor_tail_bits > 0; else 0)                  */
    int64_t u_tail_entries;  /* their U entries, sum (k_b - k32_b) |tau_b|        */
    int64_t lr_tail_entries; /* their factor entries, sum (k_b - k32_b)(|tau|+|sigma|) */
} hm_matrix_info;

/* Build the Morton-ordered cluster tree and the block cluster tree of a
 * triangle mesh (Sec. 2.3, Algorithm 1, Eq. 5; Sec. 3.1 "Spatial data
 * structure").
 *  d_vertices : [n_vertices][3] doubles (device), vertex coordinates.
 *  d_tris     : [n_tris][3] int32 (device), vertex indices of each flat
 *               triangle, each in [0, n_vertices).  n_tris >= 1.
 *  The nodes X_h are the triangle centroids ((v0 + v1) + v2) / 3; the Morton
 *  code quantises them on a 2^21 grid over the cube of side max extent; ties
 *  are ordered by original index; clusters are halved by cardinality
 *  (|tau_1| = floor(|tau| / 2)) until |tau| <= leaf_size.
 *  Errors: HM_EINVAL for NULL pointers, n_tris < 1, n_vertices < 3,
 *  n_tris > 2^28, a vertex index out of range, eta < 0 or leaf_size out of
 *  [1, 254]. */
HM_API hm_status hm_build_tree(const double *d_vertices, int64_t n_vertices, const int32_t *d_tris, int64_t n_tris,
                        const hm_tree_params *params, hm_stream_t stream, hm_tree **out);

/* Assemble the H-matrix approximation of the Galerkin matrix
 * a_ij = int_Ti int_Tj 1/(4 pi |x - y|) dsigma_y dsigma_x (Eq. 4, Sec. 3.3):
 * every non-admissible leaf is evaluated densely (7x7 tensor of the
 * degree-5 7-point rule for disjoint panels, Sauter-Schwab regularised
 * Gauss-Legendre of order ss_order for panels sharing a vertex or an edge,
 * Sec. 4.1), every admissible leaf is compressed by ACA with partial pivoting
 * to relative tolerance aca_eps with entries evaluated on the fly (Sec. 2.3).
 *  Errors: HM_EINVAL for bad parameters, HM_ENOMEM when the matrix does not
 *  fit in device memory. */
HM_API hm_status hm_assemble(const hm_tree *tree, const hm_assemble_params *params, hm_stream_t stream,
                      hm_matrix **out);

/* The trees of many independent geometries in one structure (batched
 * problems): geometry g is the triangle range [h_tri_offsets[g],
 * h_tri_offsets[g + 1]) of d_tris (indices into the shared d_vertices).  Each
 * geometry gets its own bounding cube and Morton order (the panels of a
 * geometry stay contiguous, geometries in input order), its own cluster tree
 * (cardinality halving from its own root), and Algorithm 1 runs from every
 * (root_g, root_g) pair, so no block couples two geometries: the assembled
 * operator is block diagonal and every later call (assembly, products,
 * solves) treats all geometries in the same launches.  A batched solve
 * (hm_solve_params.batched) runs one GMRES per geometry and right-hand side.
 *  h_tri_offsets: host, n_geom + 1 entries, 0 = first, n_tris = last, each
 *  geometry non-empty.  Other arguments and errors as hm_build_tree. */
HM_API hm_status hm_build_forest(const double *d_vertices, int64_t n_vertices, const int32_t *d_tris, int64_t n_tris,
                                 const int64_t *h_tri_offsets, int32_t n_geom, const hm_tree_params *params,
                                 hm_stream_t stream, hm_tree **out);

/* Load vectors of a forest with sources per geometry: d_sources is
 * [n_geom][n_per_geom][3] (device); d_f[s][i] = int_Ti 1/(4 pi |x - p_{g,s}|)
 * with g the geometry of panel i, [n_per_geom][n] in original order.
 * Errors: HM_EINVAL for NULL pointers or n_per_geom < 1. */
HM_API hm_status hm_load_vector_geom(const hm_tree *tree, const double *d_sources, int32_t n_per_geom, double *d_f,
                                     hm_stream_t stream);

/* Galerkin load vector for point-source Dirichlet data (Sec. 2.2):
 * f[s][i] = int_Ti g_s dsigma with g_s(x) = 1 / (4 pi |x - p_s|), by the
 * 7-point rule.
 *  d_sources : [n_sources][3] doubles (device).
 *  d_f       : [n_sources][n] doubles (device), original panel order.
 *  Errors: HM_EINVAL for NULL pointers or n_sources < 1. */
HM_API hm_status hm_load_vector(const hm_tree *tree, const double *d_sources, int32_t n_sources, double *d_f,
                         hm_stream_t stream);

/* Single-layer potential of a piecewise-constant density at points off the
 * surface: the ansatz U(x) = int_Gamma u(y) / (4 pi |x - y|) dsigma_y of
 * Sec. 2.1, which Sec. 4.3 evaluates at interior points to measure the
 * error; 7-point rule on every panel (the points must not lie on the
 * surface: no singular treatment).
 *  trans = 0: d_out[k] = sum_j |T_j| sum_q w_q G(p_k, y_q^j) d_in[j]
 *             (d_in: [n] density, original panel order; d_out: [n_points]);
 *  trans = 1: d_out[j] = |T_j| sum_q w_q sum_k G(p_k, y_q^j) d_in[k], the
 *             adjoint (d_in: [n_points]; d_out: [n], original order).
 *  d_points : [n_points][3] doubles (device).  All pointers device,
 *  caller-owned.  Errors: HM_EINVAL for NULL pointers or n_points < 0. */
HM_API hm_status hm_potential(const hm_tree *tree, const double *d_points, int64_t n_points, int32_t trans,
                              const double *d_in, double *d_out, hm_stream_t stream);

/* H-matrix-vector product (Sec. 2.3): y = alpha * op(H) x + beta * y, with
 * op(H) = H (trans = 0) or H^T (trans = 1), applied column by column to nrhs
 * right-hand sides stored as [nrhs][n] (original panel order).
 *  prec : HM_F64 uses the FP64 master; HM_F32 / HM_BF16 use the
 *         low-precision copies (FP32 accumulation; they must have been
 *         requested in hm_assemble).
 *  d_x, d_y : device pointers, must not overlap.
 *  trans = 1 applies the stored H transposed, as the adjoint of the product
 *  (U and W exchange roles, the near field is read transposed); the first
 *  transposed call on a matrix builds and keeps the transposed near field
 *  (one more copy of it) and its index maps, synchronising the stream once.
 *  Stream-ordered: the call queues the work on `stream` and returns; its
 *  working vectors come from the stream-ordered pool (cudaMallocAsync).
 *  Errors: HM_EINVAL for NULL pointers, nrhs < 1, a precision whose copy was
 *  not assembled, or trans not in {0, 1}. */
HM_API hm_status hm_matvec(const hm_matrix *A, int32_t trans, int32_t nrhs, hm_dtype prec, const double *d_x, double *d_y,
                    double alpha, double beta, hm_stream_t stream);

/* The product with many right-hand sides (the multi-RHS form of the
 * H-matvec of Sec. 2.3): y = alpha H x + beta y for nrhs right-hand sides
 * [nrhs][n] (original order), 16 at a time, each stored entry read once per
 * 16.
 *  prec = HM_F32 (FP32 near field and factors) or HM_BF16 (FP32 near field,
 *  BF16 factors): on the tensor cores.  The operands are BF16 (mma m16n8k16,
 *  FP32 accumulation): FP32 values, including x, are split into a BF16 pair
 *  (hi + lo) and multiplied as hi*hi + hi*lo + lo*hi, so the result carries
 *  about 16 significant bits (relative error ~1e-5 on top of the copy's own
 *  rounding) — accurate enough for the inner solves of the refinement.
 *  prec = HM_F64: the FP64 master in double-float arithmetic on the FP32
 *  pipe (every entry and x split into a pair of floats, error-free products
 *  and sums: the compensated dot product of Ogita, Rump and Oishi), about
 *  2^-47 relative error per term, ~1e-14 of the row sums of |H||x| — the
 *  FP64 residuals of the batched refinement (hm_solve_params.resid_df).
 * Stream-ordered (working vectors from the stream-ordered pool; HM_F64 uses
 * 128 bytes per panel, per partial projection and per unit of total rank).
 * Errors: HM_EINVAL for NULL pointers, nrhs < 1, an unknown precision, or a
 * low precision whose copy was not assembled. */
HM_API hm_status hm_matvec_block(const hm_matrix *A, int32_t nrhs, hm_dtype prec, const double *d_x, double *d_y,
                                 double alpha, double beta, hm_stream_t stream);

/* The H-matrix-vector product of hm_matvec (trans = 0 only) for callers that
 * must not allocate device memory during the call: code running under a fixed
 * device-memory budget or its own pool, where a cudaMalloc / cudaFree would
 * fail, block or break the caller's accounting.  The paper has no counterpart;
 * this is a property of the library interface only.
 *  Same arguments and results as hm_matvec.  Its working vectors (x and y in
 *  Morton order, the low-rank projections, and their FP32 roundings for the
 *  low-precision copies) live in one 16 MiB array that
 *  the library reserves on every device it is loaded on, held until exit; no
 *  memory is allocated or freed by the call.
 *  Limit: 2 n + K + P doubles plus n + K + P floats must fit in 2,097,152
 *  doubles (K = sum of the ACA ranks, P = the column-cluster partials of the
 *  low-rank projections of the forward product, about K times the mean
 *  number of leaf clusters an admissible block spans); larger problems get
 *  HM_EINVAL with the required size in hm_last_error().  trans = 1 is
 *  rejected with HM_EINVAL.
 *  The first call on a device looks up that array's device address (with the
 *  device current); make that first call before any stream capture.  The
 *  address is looked up again when the device's context has changed since
 *  (a cudaDeviceReset makes a new one).
 *  All calls share the array and it keeps the last call's contents: calls
 *  whose work overlaps on the GPU (different streams or host threads) race.
 *  The call is stream-ordered and does not synchronise; d_y is complete when
 *  `stream` reaches the end of the call's work. */
HM_API hm_status hm_matvec_noalloc(const hm_matrix *A, int32_t trans, int32_t nrhs, hm_dtype prec, const double *d_x,
                                   double *d_y, double alpha, double beta, hm_stream_t stream);

/* Solve op(H) x = b with restarted GMRES (Sec. 4.1 solves with a Krylov
 * method; GMRES(m) with classical Gram-Schmidt applied twice, Givens
 * rotations and the Hessenberg least-squares problem in FP64), optionally as
 * FP64 iterative refinement around a low-precision inner operator.
 *  d_b : [nrhs][n] right-hand sides (device, original order).
 *  d_x : [nrhs][n] solutions (device); the initial guess is zero.
 *  info: host pointer, may be NULL; filled for the last right-hand side.
 *  trans = 1 solves H^T x = b (the adjoint system of a gradient), with the
 *  transposed product of hm_matvec and, when precond = 1, the transposed
 *  block-Jacobi inverses.
 *  Returns HM_ENOCONV (with the best x stored) when max_iter is reached. */
HM_API hm_status hm_solve(const hm_matrix *A, int32_t trans, int32_t nrhs, const double *d_b, double *d_x,
                   const hm_solve_params *params, hm_stream_t stream, hm_solve_info *info);

/* Solves the system of the column-scaled operator A(c) = H diag(c): op(A(c)) x = b,
 * i.e. H diag(c) x = b (trans = 0) or diag(c) H^T x = b (trans = 1).  With
 * u_j = c_j x_j the density of panel j, A(c) x is the Galerkin single-layer
 * operator (Sec. 2.2, Eq. 4) applied to a density whose panel values are
 * scaled by c: the parametrisation whose gradient with respect to c the
 * adjoint method needs.  The scaling is applied by the library (trans = 0:
 * H y = b is solved, then x = y / c; trans = 1: H^T x = b / c is solved).
 *  d_c : [n] per-panel coefficients (device, original order), all nonzero
 *        (not checked: a zero gives inf / NaN entries).
 *  Other arguments, results and errors as hm_solve (the batched form is for
 *  trans = 0); on HM_ENOCONV the best x is scaled and returned too. */
HM_API hm_status hm_solve_scaled(const hm_matrix *A, int32_t trans, int32_t nrhs, const double *d_c, const double *d_b,
                                 double *d_x, const hm_solve_params *params, hm_stream_t stream, hm_solve_info *info);

/* The product with diagonal scalings on both sides:
 *   y = alpha * diag(l) op(H) diag(r) x + beta * y
 * for nrhs right-hand sides [nrhs][n] (original order; op as in hm_matvec).
 * d_left (l) and d_right (r) are [n] device vectors, each NULL for the
 * identity.  Products of the column-scaled operator A(c) = H diag(c) take
 * d_right = c (A(c) x) or d_left = c with trans = 1 (A(c)^T x); the
 * gradient of a solution functional with respect to c,
 * dL/dc_j = -alpha_j (H^T lam)_j, takes trans = 1, d_left = alpha, x = lam,
 * alpha = -1.  Stream-ordered (working vectors from the stream-ordered pool).
 * Errors as hm_matvec. */
HM_API hm_status hm_matvec_scaled(const hm_matrix *A, int32_t trans, int32_t nrhs, hm_dtype prec, const double *d_left,
                                  const double *d_right, const double *d_x, double *d_y, double alpha, double beta,
                                  hm_stream_t stream);

/* Frees an hm_tree or hm_matrix handle (NULL is a no-op).  Device buffers of
 * 1 MiB or more are not unmapped but kept by the library for its later
 * allocations (unmapping costs ~0.4 ms per GB), up to a quarter of the
 * device memory; the library empties that cache by itself when one of its
 * own allocations fails. */
HM_API void hm_free(void *handle);

/* Adds a low-precision copy to an assembled matrix, made from its FP64
 * master and kept with it: dtype HM_F32 = FP32 copies of the near field and
 * the factors; HM_BF16 = BF16 factors (and the FP32 near field they run
 * with).  A copy that exists is kept as it is.  Afterwards the matrix serves
 * products and inner solves in that precision exactly as if the assembly had
 * kept the copy (the same rounding of the same FP64 values).  Stream-ordered.
 * HM_EINVAL for another dtype, HM_ENOMEM when it does not fit. */
HM_API hm_status hm_matrix_add_copy(const hm_matrix *A, hm_dtype dtype, hm_stream_t stream);

/* Returns every device block the library keeps for reuse to the driver
 * (for callers that need the memory for other allocations).  Synchronises
 * the device. */
HM_API void hm_trim(void);

/* Limit, in SM clock cycles, of the library's bounded device-side waits
 * (the wait of the near-field assembly for its TMA-staged panel tiles, and
 * the mbarrier waits of the tcgen05 row pass of the 16-right-hand-side
 * product, hm_assemble_params.mrhs_tcgen05), for the calls that follow,
 * from any thread.  cycles >= 0 sets it; cycles < 0
 * restores the default of 4e9 cycles (about 2 s at 2 GHz).  A wait that
 * reaches the limit records the failure and makes the call return
 * HM_ETIMEOUT; before its thread block exits it waits again, with the
 * default limit, for the copies it started, so that no copy lands in shared
 * memory after the block has left (the tcgen05 row pass likewise waits for
 * its MMAs and copies before it frees its tensor memory).  0 gives up before
 * the first poll: every assembly with dense leaves, and every product
 * through the tcgen05 row pass, then returns HM_ETIMEOUT (a hook for testing
 * those paths).  After HM_ETIMEOUT the assembly's matrix is not created (a
 * product's output is undefined) and the device context stays usable; if the second, default-limit wait also
 * gave up (a copy that never completed) the context should be treated as
 * suspect.  The paper has no counterpart.  Always HM_OK. */
HM_API hm_status hm_set_wait_limit(int64_t cycles);

/* Injected allocation failure, for testing the error paths: with n > 0 the
 * n-th device allocation the library makes from now on (from any thread)
 * fails as an exhausted cudaMalloc would, so the call that makes it returns
 * HM_ENOMEM, releasing what it had allocated; the injection then disarms
 * itself.  n = 0 disarms it.  The environment variable HM_FAULT_INJECT=<n>
 * arms it when the library is loaded.  The paper has no counterpart.
 * Always HM_OK. */
HM_API hm_status hm_set_fault_injection(int64_t n);

/* Measured FMA throughput of the current device, in TFLOP/s (an FMA counts
 * 2 flops): kind = HM_F64 (DFMA) or HM_F32 (FFMA).  A kernel fills every SM
 * with threads that each run eight independent FMA chains; the best of three
 * timed launches (after one warm-up launch, CUDA events on `stream`, about
 * 20-50 ms each) is returned.  The paper has no counterpart: the figures are
 * the denominators of the ALU rooflines of this library's kernels (the
 * nominal FP64 rate of unit counts x clock is above what this part's FP64
 * pipe delivers).  The result depends on the SM clock during the call.
 * Synchronises the stream.  Errors: HM_EINVAL for a NULL pointer or another
 * kind. */
HM_API hm_status hm_measure_fma_peak(hm_dtype kind, double *tflops, hm_stream_t stream);

/* Tree introspection (synchronises the stream of the tree). */
HM_API hm_status hm_tree_get_info(const hm_tree *tree, hm_tree_info *info);

/* d_perm[k] = original index of the panel at Morton position k ([n] int32,
 * device). */
HM_API hm_status hm_tree_get_perm(const hm_tree *tree, int32_t *d_perm);

/* Leaves of the block tree as [count][4] int32 (row_begin, row_end,
 * col_begin, col_end) in Morton positions, written to d_out (device) when
 * capacity >= count; *count always receives the number of leaves.
 * dense = 1: non-admissible leaves; dense = 0: admissible leaves. */
HM_API hm_status hm_tree_get_leaves(const hm_tree *tree, int32_t dense, int32_t *d_out, int64_t capacity, int64_t *count);

HM_API hm_status hm_matrix_get_info(const hm_matrix *A, hm_matrix_info *info);

/* Copies the FP64 H-matrix to host memory in a plain layout, so that it can be
 * re-applied independently:
 *  dense leaves b = 0..n_dense-1 in the order of hm_tree_get_leaves(dense=1):
 *     h_dense[h_dense_off[b] + i * n_b + j] = a(row_begin + i, col_begin + j)
 *  admissible leaves b = 0..n_adm-1 in the order of hm_tree_get_leaves(dense=0):
 *     rank h_rank[b]; U_b (m_b x k_b, column-major) at h_uw + h_u_off[b];
 *     W_b (n_b x k_b, column-major) at h_uw + h_w_off[b]; block ~ U_b W_b^T.
 * Pass NULL value pointers to query the sizes only: *n_dense_vals and
 * *n_lr_vals receive the element counts of h_dense and h_uw. */
HM_API hm_status hm_matrix_export(const hm_matrix *A, double *h_dense, int64_t *h_dense_off, int32_t *h_rank, double *h_uw,
                           int64_t *h_u_off, int64_t *h_w_off, int64_t *n_dense_vals, int64_t *n_lr_vals);

/* Number of CUDA kernels this library has launched since it was loaded (all
 * threads).  Lets a caller count the device work behind a sequence of calls. */
HM_API int64_t hm_kernel_launches(void);

/* Kernel timing trace.  hm_trace_enable(1) clears the trace and starts it;
 * while it runs, the library brackets each launch of its main kernels (the
 * near-field, touching-pair and ACA kernels, the three kernels of the
 * H-matvec per precision, and the solver's block-Jacobi, dot-product and
 * update kernels) with a pair of CUDA events recorded on the launching stream
 * (not while that stream is being captured).  hm_trace_enable(0) stops it and
 * keeps what was recorded.  The library has no counterpart in the paper; it
 * exists so that a caller can time single kernels inside a longer sequence. */
HM_API hm_status hm_trace_enable(int32_t on);

typedef struct {
    char name[48];    /* kernel name, with ".f64" / ".f32" / ".bf16" for the matvec */
    int64_t launches; /* traced launches                                            */
    double ms;        /* summed device time of those launches, milliseconds         */
} hm_trace_entry;

/* Per-kernel totals of the trace: up to `capacity` entries into out (host),
 * *count receives the number of distinct kernels.  Waits for the recorded
 * events.  Errors: HM_EINVAL for NULL count, HM_ECUDA for a failed event. */
HM_API hm_status hm_trace_read(hm_trace_entry *out, int32_t capacity, int32_t *count);

/* One leaf of the H-matrix as a dense row-major m x n array written to d_out
 * (device, caller-owned, m * n doubles): the stored entries of a
 * non-admissible leaf (dense = 1), or the product U_b W_b^T of an admissible
 * leaf (dense = 0); `index` as in hm_tree_get_leaves.  Introspection for
 * checks on large problems, where hm_matrix_export would not fit in host
 * memory.  Errors: HM_EINVAL for a bad handle, index or NULL pointer. */
HM_API hm_status hm_matrix_get_block(const hm_matrix *A, int32_t dense, int64_t index, double *d_out,
                                     hm_stream_t stream);

/* Message of the last failure on the calling thread ("" when none). */
HM_API const char *hm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HM_H */
