/*
 * hm_oracle.c -- plain, slow FP64 CPU oracle of the H-matrix BEM hot path of
 * Harbrecht & Zaspel, "A scalable H-matrix approach for the solution of
 * boundary integral equations on multi-GPU clusters" (arXiv 1806.11558).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark load this library; the product (CUDA) path never
 * does, and the two share no code, headers or tables.
 *
 * Compiled with -O2 -ffp-contract=off: every floating-point operation below is
 * one correctly rounded IEEE operation, evaluated in the order written.
 * OpenMP (when enabled) only distributes independent rows / blocks over
 * threads; it never reorders the arithmetic of one entry or one block.
 *
 * What is computed (paper section in brackets):
 *   - the single-layer Laplace kernel G(x,y) = 1/(4 pi |x-y|)      [Sec. 2.1, Example 2.1]
 *   - Galerkin entries a_ij = int_Ti int_Tj G dsigma_y dsigma_x    [Sec. 2.2, Eq. 4]
 *     with piecewise-constant (P0) basis on flat triangles          [Sec. 4.1]
 *       * regular pairs (no shared vertex): 7x7 tensor of the
 *         degree-5 7-point triangle rule
 *       * touching pairs: Sauter-Schwab / Duffy regularising
 *         transformations ("Duffy trick", Sec. 4.1), with the radial
 *         variable integrated exactly and Gauss-Legendre in the rest
 *   - the load vector f_i = int_Ti g dsigma                          [Sec. 2.2]
 *   - the single-layer potential (S~ u_h)(x)                         [Sec. 2.1, Eq. 2]
 *   - the block cluster tree of Algorithm 1 under Eq. 5             [Sec. 2.3]
 *   - ACA with partial pivoting of admissible blocks                [Sec. 2.3]
 *   - the H-matrix-vector product (and its transpose)               [Sec. 2.3]
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define NQ 7

/* ------------------------------------------------------------------------ */
/* geometry helpers                                                          */
/* ------------------------------------------------------------------------ */

static void vsub(const double *a, const double *b, double *o)
{
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}

static double vnorm(const double *a)
{
    return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
}

/* |T| = |(v1 - v0) x (v2 - v0)| / 2 */
static double tri_area(const double *v0, const double *v1, const double *v2)
{
    double e1[3], e2[3], c[3];
    vsub(v1, v0, e1);
    vsub(v2, v0, e2);
    c[0] = e1[1] * e2[2] - e1[2] * e2[1];
    c[1] = e1[2] * e2[0] - e1[0] * e2[2];
    c[2] = e1[0] * e2[1] - e1[1] * e2[0];
    return 0.5 * vnorm(c);
}

static const double *vtx(const double *V, const int32_t *T, int64_t i, int k)
{
    return V + 3 * (int64_t)T[3 * i + k];
}

/* physical quadrature points x_q = b0 v0 + b1 v1 + b2 v2 */
static void quad_points(const double *V, const int32_t *T, int64_t i, const double *bary, double x[NQ][3])
{
    const double *a = vtx(V, T, i, 0), *b = vtx(V, T, i, 1), *c = vtx(V, T, i, 2);
    for (int q = 0; q < NQ; ++q)
        for (int d = 0; d < 3; ++d)
            x[q][d] = bary[3 * q] * a[d] + bary[3 * q + 1] * b[d] + bary[3 * q + 2] * c[d];
}

/* ------------------------------------------------------------------------ */
/* regular entries: 7x7 tensor rule                                          */
/* ------------------------------------------------------------------------ */

static double entry_regular(const double *V, const int32_t *T, int64_t i, int64_t j,
                            const double *bary, const double *w7)
{
    double x[NQ][3], y[NQ][3], d[3];
    quad_points(V, T, i, bary, x);
    quad_points(V, T, j, bary, y);
    double s = 0.0;
    for (int p = 0; p < NQ; ++p) {
        double sp = 0.0;
        for (int q = 0; q < NQ; ++q) {
            vsub(x[p], y[q], d);
            sp += w7[q] / vnorm(d);
        }
        s += w7[p] * sp;
    }
    double ai = tri_area(vtx(V, T, i, 0), vtx(V, T, i, 1), vtx(V, T, i, 2));
    double aj = tri_area(vtx(V, T, j, 0), vtx(V, T, j, 1), vtx(V, T, j, 2));
    return ai * aj * s / (4.0 * M_PI);
}

/* ------------------------------------------------------------------------ */
/* Sauter-Schwab regularising transformations                                */
/*                                                                          */
/* Reference triangle  That = {(u1,u2): 0 <= u2 <= u1 <= 1},  area 1/2,       */
/* chi(u) = P0 + u1 (P1 - P0) + u2 (P2 - P1),  |det| = 2|T|.                   */
/* For a pair of touching panels the vertex lists are ordered so that the    */
/* shared vertices come first (P0 = Q0, and P1 = Q1 for a shared edge).  The  */
/* singular set is then mapped to xi = 0 of (xi, eta1, eta2, eta3) in [0,1]^4 */
/* by the regions below: 6 for identical panels, 5 for a common edge, 2 for   */
/* a common vertex.  Both (u, v) scale linearly with xi, so for flat panels   */
/* chi_P(u) - chi_Q(v) = xi * D(eta) and the kernel is 1/(4 pi xi |D|); the   */
/* Jacobian carries xi^3, so the xi-integral is exactly  int xi^2 = 1/3.      */
/* ------------------------------------------------------------------------ */

enum { SS_COINCIDENT = 3, SS_EDGE = 2, SS_VERTEX = 1 };

static int ss_nregions(int kind)
{
    return kind == SS_COINCIDENT ? 6 : (kind == SS_EDGE ? 5 : 2);
}

/* region map r of the given kind at (xi, e1, e2, e3): points u, v of That and
 * the Jacobian of (xi,e) -> (u,v). */
static void ss_map(int kind, int r, double xi, double e1, double e2, double e3,
                   double u[2], double v[2], double *jac)
{
    if (kind == SS_COINCIDENT) {
        *jac = xi * xi * xi * e1 * e1 * e2;
        switch (r) {
        case 0: u[0] = xi; u[1] = xi * (1.0 - e1 + e1 * e2);
                v[0] = xi * (1.0 - e1 * e2 * e3); v[1] = xi * (1.0 - e1); break;
        case 1: u[0] = xi * (1.0 - e1 * e2 * e3); u[1] = xi * (1.0 - e1);
                v[0] = xi; v[1] = xi * (1.0 - e1 + e1 * e2); break;
        case 2: u[0] = xi; u[1] = xi * e1 * (1.0 - e2 + e2 * e3);
                v[0] = xi * (1.0 - e1 * e2); v[1] = xi * e1 * (1.0 - e2); break;
        case 3: u[0] = xi * (1.0 - e1 * e2); u[1] = xi * e1 * (1.0 - e2);
                v[0] = xi; v[1] = xi * e1 * (1.0 - e2 + e2 * e3); break;
        case 4: u[0] = xi * (1.0 - e1 * e2 * e3); u[1] = xi * e1 * (1.0 - e2 * e3);
                v[0] = xi; v[1] = xi * e1 * (1.0 - e2); break;
        default: u[0] = xi; u[1] = xi * e1 * (1.0 - e2);
                 v[0] = xi * (1.0 - e1 * e2 * e3); v[1] = xi * e1 * (1.0 - e2 * e3); break;
        }
    } else if (kind == SS_EDGE) {
        switch (r) {
        case 0: *jac = xi * xi * xi * e1 * e1;
                u[0] = xi; u[1] = xi * e1 * e3;
                v[0] = xi * (1.0 - e1 * e2); v[1] = xi * e1 * (1.0 - e2); break;
        case 1: *jac = xi * xi * xi * e1 * e1 * e2;
                u[0] = xi; u[1] = xi * e1;
                v[0] = xi * (1.0 - e1 * e2 * e3); v[1] = xi * e1 * e2 * (1.0 - e3); break;
        case 2: *jac = xi * xi * xi * e1 * e1 * e2;
                u[0] = xi * (1.0 - e1 * e2); u[1] = xi * e1 * (1.0 - e2);
                v[0] = xi; v[1] = xi * e1 * e2 * e3; break;
        case 3: *jac = xi * xi * xi * e1 * e1 * e2;
                u[0] = xi * (1.0 - e1 * e2 * e3); u[1] = xi * e1 * e2 * (1.0 - e3);
                v[0] = xi; v[1] = xi * e1; break;
        default: *jac = xi * xi * xi * e1 * e1 * e2;
                 u[0] = xi * (1.0 - e1 * e2 * e3); u[1] = xi * e1 * (1.0 - e2 * e3);
                 v[0] = xi; v[1] = xi * e1 * e2; break;
        }
    } else {
        *jac = xi * xi * xi * e2;
        if (r == 0) {
            u[0] = xi; u[1] = xi * e1;
            v[0] = xi * e2; v[1] = xi * e2 * e3;
        } else {
            u[0] = xi * e2; u[1] = xi * e2 * e3;
            v[0] = xi; v[1] = xi * e1;
        }
    }
}

/* Order the vertices of touching panels i, j so that shared ones come first.
 * Common edge: the shared pair in the order it appears in T_i.  Common
 * vertex: each panel's vertices cyclically rotated to start at the shared one.
 * Returns the number of shared vertices (0 = regular pair). */
static int touch_order(const int32_t *T, int64_t i, int64_t j, int32_t P[3], int32_t Q[3])
{
    const int32_t *ti = T + 3 * i, *tj = T + 3 * j;
    int in_j[3], nshared = 0;
    for (int a = 0; a < 3; ++a) {
        in_j[a] = -1;
        for (int b = 0; b < 3; ++b)
            if (ti[a] == tj[b]) in_j[a] = b;
        if (in_j[a] >= 0) ++nshared;
    }
    if (nshared == 3) {
        for (int a = 0; a < 3; ++a) { P[a] = ti[a]; Q[a] = ti[a]; }
    } else if (nshared == 2) {
        int k = 0;
        for (int a = 0; a < 3; ++a)
            if (in_j[a] >= 0) { P[k] = ti[a]; Q[k] = ti[a]; ++k; }
        for (int a = 0; a < 3; ++a)
            if (in_j[a] < 0) P[2] = ti[a];
        for (int b = 0; b < 3; ++b)
            if (tj[b] != P[0] && tj[b] != P[1]) Q[2] = tj[b];
    } else if (nshared == 1) {
        int a0 = 0;
        for (int a = 0; a < 3; ++a)
            if (in_j[a] >= 0) a0 = a;
        int b0 = in_j[a0];
        for (int k = 0; k < 3; ++k) {
            P[k] = ti[(a0 + k) % 3];
            Q[k] = tj[(b0 + k) % 3];
        }
    }
    return nshared;
}

static double entry_singular(const double *V, int kind, const int32_t P[3], const int32_t Q[3],
                             int ngl, const double *xgl, const double *wgl)
{
    const double *p0 = V + 3 * (int64_t)P[0], *p1 = V + 3 * (int64_t)P[1], *p2 = V + 3 * (int64_t)P[2];
    const double *q0 = V + 3 * (int64_t)Q[0], *q1 = V + 3 * (int64_t)Q[1], *q2 = V + 3 * (int64_t)Q[2];
    double a1[3], a2[3], b1[3], b2[3];
    vsub(p1, p0, a1);
    vsub(p2, p1, a2);
    vsub(q1, q0, b1);
    vsub(q2, q1, b2);
    int nr = ss_nregions(kind);
    double s = 0.0;
    for (int r = 0; r < nr; ++r)
        for (int k1 = 0; k1 < ngl; ++k1)
            for (int k2 = 0; k2 < ngl; ++k2)
                for (int k3 = 0; k3 < ngl; ++k3) {
                    double u[2], v[2], jac, d[3];
                    ss_map(kind, r, 1.0, xgl[k1], xgl[k2], xgl[k3], u, v, &jac);
                    for (int c = 0; c < 3; ++c)
                        d[c] = (u[0] * a1[c] + u[1] * a2[c]) - (v[0] * b1[c] + v[1] * b2[c]);
                    s += wgl[k1] * wgl[k2] * wgl[k3] * jac / vnorm(d);
                }
    double ai = tri_area(p0, p1, p2), aj = tri_area(q0, q1, q2);
    /* 4|Ti||Tj| from the two parametrisations, 1/3 from the xi-integral */
    return 4.0 * ai * aj * (s / 3.0) / (4.0 * M_PI);
}

/* a_ij for original panel indices i, j */
double orc_entry(const double *V, const int32_t *T, int64_t i, int64_t j,
                 const double *bary, const double *w7, int ngl, const double *xgl, const double *wgl)
{
    int32_t P[3], Q[3];
    int ns = touch_order(T, i, j, P, Q);
    if (ns == 0) return entry_regular(V, T, i, j, bary, w7);
    return entry_singular(V, ns, P, Q, ngl, xgl, wgl);
}

/* number of shared vertices of panels i and j (0..3) */
int orc_touch(const int32_t *T, int64_t i, int64_t j)
{
    int32_t P[3], Q[3];
    return touch_order(T, i, j, P, Q);
}

/* Region maps evaluated at npts points, for every region of `kind`; output
 * u, v as [region][pt][2] and jac as [region][pt].  Used by the tests that
 * check that the regions tile That x That exactly. */
void orc_ss_points(int kind, int64_t npts, const double *xi, const double *e1, const double *e2,
                   const double *e3, double *u, double *v, double *jac)
{
    int nr = ss_nregions(kind);
    for (int r = 0; r < nr; ++r)
        for (int64_t k = 0; k < npts; ++k)
            ss_map(kind, r, xi[k], e1[k], e2[k], e3[k], u + 2 * (r * npts + k), v + 2 * (r * npts + k),
                   jac + r * npts + k);
}

/* Dense sub-matrix out[a][b] = a_{rows[a], cols[b]} (original indices). */
void orc_assemble(const double *V, const int32_t *T, int64_t nr, const int64_t *rows, int64_t nc,
                  const int64_t *cols, const double *bary, const double *w7, int ngl, const double *xgl,
                  const double *wgl, double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < nr; ++a)
        for (int64_t b = 0; b < nc; ++b)
            out[a * nc + b] = orc_entry(V, T, rows[a], cols[b], bary, w7, ngl, xgl, wgl);
}

/* Load vector for point sources: f[s][i] = |T_i| sum_q w_q / (4 pi |x_q - p_s|). */
void orc_load_vector(const double *V, const int32_t *T, int64_t n, const double *bary, const double *w7,
                     int64_t nsrc, const double *src, double *f)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double x[NQ][3], d[3];
        quad_points(V, T, i, bary, x);
        double ai = tri_area(vtx(V, T, i, 0), vtx(V, T, i, 1), vtx(V, T, i, 2));
        for (int64_t s = 0; s < nsrc; ++s) {
            double acc = 0.0;
            for (int q = 0; q < NQ; ++q) {
                vsub(x[q], src + 3 * s, d);
                acc += w7[q] / vnorm(d);
            }
            f[s * n + i] = ai * acc / (4.0 * M_PI);
        }
    }
}

/* Single-layer potential of a P0 density: out[k] = sum_j alpha_j int_Tj G(x_k, y) dsigma_y,
 * with the 7-point rule on every panel (the evaluation points lie off the surface). */
void orc_potential(const double *V, const int32_t *T, int64_t n, const double *alpha, const double *bary,
                   const double *w7, int64_t npts, const double *pts, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npts; ++k) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double y[NQ][3], d[3];
            quad_points(V, T, j, bary, y);
            double s = 0.0;
            for (int q = 0; q < NQ; ++q) {
                vsub(pts + 3 * k, y[q], d);
                s += w7[q] / vnorm(d);
            }
            acc += alpha[j] * tri_area(vtx(V, T, j, 0), vtx(V, T, j, 1), vtx(V, T, j, 2)) * s;
        }
        out[k] = acc / (4.0 * M_PI);
    }
}

/* E[k][j] = |T_j| sum_q w_q / (4 pi |p_k - y_q^j|): the single-layer potential
 * of Sec. 2.1 at point p_k of the j-th basis function (indicator of T_j), so
 * that (S~ u_h)(p_k) = sum_j E[k][j] alpha_j.  Row-major [npts][n]. */
void orc_potential_matrix(const double *V, const int32_t *T, int64_t n, const double *bary, const double *w7,
                          int64_t npts, const double *pts, double *E)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npts; ++k) {
        for (int64_t j = 0; j < n; ++j) {
            double y[NQ][3], d[3];
            quad_points(V, T, j, bary, y);
            double s = 0.0;
            for (int q = 0; q < NQ; ++q) {
                vsub(pts + 3 * k, y[q], d);
                s += w7[q] / vnorm(d);
            }
            E[k * n + j] = tri_area(vtx(V, T, j, 0), vtx(V, T, j, 1), vtx(V, T, j, 2)) * s / (4.0 * M_PI);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Block cluster tree: Algorithm 1 with the admissibility condition Eq. 5     */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *c;      /* centroids in Morton order, [N][3] */
    int64_t leaf;
    double eta2;
    int64_t nd, na, cap;
    int64_t *dense, *adm; /* [cap][4] */
    int overflow;
} btree_t;

/* Q_tau: componentwise min / max of the centroids in [b, e) */
static void cluster_box(const double *c, int64_t b, int64_t e, double lo[3], double hi[3])
{
    for (int d = 0; d < 3; ++d) { lo[d] = c[3 * b + d]; hi[d] = c[3 * b + d]; }
    for (int64_t k = b + 1; k < e; ++k)
        for (int d = 0; d < 3; ++d) {
            if (c[3 * k + d] < lo[d]) lo[d] = c[3 * k + d];
            if (c[3 * k + d] > hi[d]) hi[d] = c[3 * k + d];
        }
}

/* Eq. 5 in squared form: min(diam^2) <= eta^2 dist^2 */
int orc_admissible(const double *lt, const double *ht, const double *ls, const double *hs, double eta2)
{
    double dt[3], ds[3], g[3];
    for (int d = 0; d < 3; ++d) {
        dt[d] = ht[d] - lt[d];
        ds[d] = hs[d] - ls[d];
        double g1 = ls[d] - ht[d], g2 = lt[d] - hs[d];
        g[d] = 0.0;
        if (g1 > g[d]) g[d] = g1;
        if (g2 > g[d]) g[d] = g2;
    }
    double diam2_t = dt[0] * dt[0] + dt[1] * dt[1] + dt[2] * dt[2];
    double diam2_s = ds[0] * ds[0] + ds[1] * ds[1] + ds[2] * ds[2];
    double dist2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    double mind = diam2_t < diam2_s ? diam2_t : diam2_s;
    return mind <= eta2 * dist2;
}

static void push(int64_t *arr, int64_t *n, int64_t cap, int *overflow, int64_t rb, int64_t re, int64_t cb, int64_t ce)
{
    if (*n >= cap) { *overflow = 1; return; }
    arr[4 * *n] = rb; arr[4 * *n + 1] = re; arr[4 * *n + 2] = cb; arr[4 * *n + 3] = ce;
    ++*n;
}

static void build_block(btree_t *t, int64_t rb, int64_t re, int64_t cb, int64_t ce)
{
    double lt[3], ht[3], ls[3], hs[3];
    cluster_box(t->c, rb, re, lt, ht);
    cluster_box(t->c, cb, ce, ls, hs);
    int adm = orc_admissible(lt, ht, ls, hs, t->eta2);
    if (!adm && re - rb > t->leaf && ce - cb > t->leaf) {
        /* cardinality-based split: |tau_1| = floor(|tau| / 2) */
        int64_t rm = rb + (re - rb) / 2, cm = cb + (ce - cb) / 2;
        build_block(t, rb, rm, cb, cm);
        build_block(t, rb, rm, cm, ce);
        build_block(t, rm, re, cb, cm);
        build_block(t, rm, re, cm, ce);
    } else if (adm) {
        push(t->adm, &t->na, t->cap, &t->overflow, rb, re, cb, ce);
    } else {
        push(t->dense, &t->nd, t->cap, &t->overflow, rb, re, cb, ce);
    }
}

/* Runs Algorithm 1 from I x I.  Leaves are (row_begin, row_end, col_begin,
 * col_end) in Morton positions.  Returns 0, or -1 if cap was too small. */
int orc_block_tree(int64_t n, const double *cent_sorted, int64_t leaf, double eta, int64_t cap,
                   int64_t *dense, int64_t *nd, int64_t *adm, int64_t *na)
{
    btree_t t;
    t.c = cent_sorted; t.leaf = leaf; t.eta2 = eta * eta;
    t.nd = 0; t.na = 0; t.cap = cap; t.dense = dense; t.adm = adm; t.overflow = 0;
    if (n > 0) build_block(&t, 0, n, 0, n);
    *nd = t.nd;
    *na = t.na;
    return t.overflow ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* ACA with partial pivoting (Sec. 2.3; Bebendorf 2000/2003)                 */
/* ------------------------------------------------------------------------ */

/* entry source of a block: returns B(i, j) for local indices */
typedef double (*entry_fn)(const void *ctx, int64_t i, int64_t j);

typedef struct {
    const double *V; const int32_t *T; const int32_t *perm;
    const double *bary, *w7, *xgl, *wgl; int ngl;
    int64_t rb, cb;
} mesh_block;

static double mesh_block_entry(const void *ctx, int64_t i, int64_t j)
{
    const mesh_block *e = (const mesh_block *)ctx;
    return orc_entry(e->V, e->T, e->perm[e->rb + i], e->perm[e->cb + j], e->bary, e->w7, e->ngl, e->xgl, e->wgl);
}

typedef struct { const double *B; int64_t n; } dense_block;

static double dense_block_entry(const void *ctx, int64_t i, int64_t j)
{
    const dense_block *d = (const dense_block *)ctx;
    return d->B[i * d->n + j];
}

/* ACA with partial pivoting of an m x n block given entry-wise.
 *  1. i_1 = row 0; no rows / columns used; ||S_0||^2 = 0.
 *  2. residual row  ~u = B(i_r, :) - sum_{l<r} U(i_r, l) W(:, l)^T;
 *     column pivot  j_r = argmax over unused columns of |~u_j| (lowest j on ties);
 *     delta = ~u(j_r).
 *  3. zero row (delta == 0 for r = 1, |delta| <= 2^-50 |delta_1| after): mark
 *     i_r used, retry with the lowest unused row without counting the step.
 *  4. W(:, r) = ~u / delta;  U(:, r) = B(:, j_r) - sum_{l<r} W(j_r, l) U(:, l).
 *  5. ||S_r||^2 = ||S_{r-1}||^2 + 2 sum_{l<r} (u_r.u_l)(w_l.w_r) + ||u_r||^2 ||w_r||^2.
 *  6. stop when ||u_r|| ||w_r|| <= eps ||S_r||, or r = min(m, n, kmax).
 *  7. next row i_{r+1} = argmax over unused rows of |u_r(i)| (lowest i on ties).
 * U column-major m x kmax (ld m), W column-major n x kmax (ld n): block ~ U W^T.
 * Optional piv_r / piv_c receive the pivot rows / columns.  Returns the rank. */
static int aca_block(entry_fn get, const void *ctx, int64_t m, int64_t n, double eps, int kmax, double *U,
                     double *W, int32_t *piv_r, int32_t *piv_c)
{
    if (m <= 0 || n <= 0) return 0;
    char *urow = calloc((size_t)m, 1), *ucol = calloc((size_t)n, 1);
    double *rowres = malloc(sizeof(double) * (size_t)n);
    int rmax = kmax;
    if (m < rmax) rmax = (int)m;
    if (n < rmax) rmax = (int)n;
    int r = 0;
    int64_t i = 0;
    double s2 = 0.0, delta1 = 0.0;
    const double tiny = ldexp(1.0, -50);
    while (r < rmax) {
        for (int64_t j = 0; j < n; ++j) {
            double v = get(ctx, i, j);
            for (int l = 0; l < r; ++l) v -= U[(int64_t)l * m + i] * W[(int64_t)l * n + j];
            rowres[j] = v;
        }
        urow[i] = 1;
        int64_t jp = -1;
        double best = -1.0;
        for (int64_t j = 0; j < n; ++j)
            if (!ucol[j] && fabs(rowres[j]) > best) { best = fabs(rowres[j]); jp = j; }
        double delta = rowres[jp];
        int zero_row = (r == 0) ? (delta == 0.0) : (fabs(delta) <= tiny * delta1);
        if (zero_row) {
            int64_t nxt = -1;
            for (int64_t k = 0; k < m; ++k)
                if (!urow[k]) { nxt = k; break; }
            if (nxt < 0) break;
            i = nxt;
            continue;
        }
        if (r == 0) delta1 = fabs(delta);
        double *ur = U + (int64_t)r * m, *wr = W + (int64_t)r * n;
        for (int64_t j = 0; j < n; ++j) wr[j] = rowres[j] / delta;
        for (int64_t k = 0; k < m; ++k) {
            double v = get(ctx, k, jp);
            for (int l = 0; l < r; ++l) v -= W[(int64_t)l * n + jp] * U[(int64_t)l * m + k];
            ur[k] = v;
        }
        ucol[jp] = 1;
        if (piv_r) piv_r[r] = (int32_t)i;
        if (piv_c) piv_c[r] = (int32_t)jp;
        double nu2 = 0.0, nw2 = 0.0;
        for (int64_t k = 0; k < m; ++k) nu2 += ur[k] * ur[k];
        for (int64_t j = 0; j < n; ++j) nw2 += wr[j] * wr[j];
        double cross = 0.0;
        for (int l = 0; l < r; ++l) {
            double du = 0.0, dw = 0.0;
            for (int64_t k = 0; k < m; ++k) du += ur[k] * U[(int64_t)l * m + k];
            for (int64_t j = 0; j < n; ++j) dw += W[(int64_t)l * n + j] * wr[j];
            cross += du * dw;
        }
        s2 = s2 + 2.0 * cross + nu2 * nw2;
        ++r;
        if (sqrt(nu2) * sqrt(nw2) <= eps * sqrt(s2)) break;
        int64_t ip = -1;
        best = -1.0;
        for (int64_t k = 0; k < m; ++k)
            if (!urow[k] && fabs(ur[k]) > best) { best = fabs(ur[k]); ip = k; }
        if (ip < 0) break;
        i = ip;
    }
    free(urow);
    free(ucol);
    free(rowres);
    return r;
}

/* ACA of every block b = (rb, re, cb, ce) in Morton positions.  Block b's
 * factors go to UW + off[b]: U (m x kmax, col-major) then W (n x kmax). */
void orc_aca_blocks(const double *V, const int32_t *T, const int32_t *perm, const double *bary, const double *w7,
                    int ngl, const double *xgl, const double *wgl, int64_t nb, const int64_t *blocks, double eps,
                    int kmax, const int64_t *off, double *UW, int32_t *rank)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nb; ++b) {
        int64_t rb = blocks[4 * b], re = blocks[4 * b + 1], cb = blocks[4 * b + 2], ce = blocks[4 * b + 3];
        int64_t m = re - rb, n = ce - cb;
        mesh_block e = {V, T, perm, bary, w7, xgl, wgl, ngl, rb, cb};
        rank[b] = aca_block(mesh_block_entry, &e, m, n, eps, kmax, UW + off[b], UW + off[b] + m * (int64_t)kmax,
                            NULL, NULL);
    }
}

/* ACA of an explicit row-major m x n matrix (used to pin the algorithm on
 * hand-built matrices).  Returns the rank; pivots go to piv_r / piv_c. */
int orc_aca_matrix(int64_t m, int64_t n, const double *B, double eps, int kmax, double *U, double *W,
                   int32_t *piv_r, int32_t *piv_c)
{
    dense_block d = {B, n};
    return aca_block(dense_block_entry, &d, m, n, eps, kmax, U, W, piv_r, piv_c);
}

/* ------------------------------------------------------------------------ */
/* H-matrix-vector product (Sec. 2.3): dense leaves apply their stored block, */
/* low-rank leaves apply U (W^T x).  trans = 1 applies H^T.                   */
/* Dense block b: row-major m x n at dval + doff[b].                          */
/* Low-rank block b: U at uw + uoff[b] (col-major, ld m), W at uw + woff[b]    */
/* (col-major, ld n), rank[b] columns.  Everything in Morton positions.       */
/* ------------------------------------------------------------------------ */
void orc_hmatvec(int trans, int64_t n, int64_t nd, const int64_t *dense, const int64_t *doff, const double *dval,
                 int64_t na, const int64_t *adm, const int32_t *rank, const int64_t *uoff, const int64_t *woff,
                 const double *uw, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
    for (int64_t b = 0; b < nd; ++b) {
        int64_t rb = dense[4 * b], re = dense[4 * b + 1], cb = dense[4 * b + 2], ce = dense[4 * b + 3];
        int64_t m = re - rb, nn = ce - cb;
        const double *A = dval + doff[b];
        for (int64_t a = 0; a < m; ++a)
            for (int64_t c = 0; c < nn; ++c) {
                if (!trans) y[rb + a] += A[a * nn + c] * x[cb + c];
                else y[cb + c] += A[a * nn + c] * x[rb + a];
            }
    }
    for (int64_t b = 0; b < na; ++b) {
        int64_t rb = adm[4 * b], re = adm[4 * b + 1], cb = adm[4 * b + 2], ce = adm[4 * b + 3];
        int64_t m = re - rb, nn = ce - cb;
        const double *U = uw + uoff[b], *W = uw + woff[b];
        for (int l = 0; l < rank[b]; ++l) {
            double t = 0.0;
            if (!trans) {
                for (int64_t c = 0; c < nn; ++c) t += W[(int64_t)l * nn + c] * x[cb + c];
                for (int64_t a = 0; a < m; ++a) y[rb + a] += U[(int64_t)l * m + a] * t;
            } else {
                for (int64_t a = 0; a < m; ++a) t += U[(int64_t)l * m + a] * x[rb + a];
                for (int64_t c = 0; c < nn; ++c) y[cb + c] += W[(int64_t)l * nn + c] * t;
            }
        }
    }
}
