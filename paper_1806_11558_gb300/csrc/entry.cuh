// entry.cuh -- device evaluation of Galerkin entries of the single-layer
// Laplace operator (Sec. 2.1 Example 2.1, Sec. 2.2 Eq. 4) for piecewise-
// constant elements on flat triangles.
//
//   a_ij = int_Ti int_Tj 1 / (4 pi |x - y|) dsigma_y dsigma_x
//
// Panels sharing no vertex: 7 x 7 tensor product of the degree-5 7-point
// triangle rule.  Panels sharing a vertex, an edge, or identical: Sauter-
// Schwab regularising transformations (the "Duffy trick" of Sec. 4.1): on
// That = {0 <= u2 <= u1 <= 1} with chi(u) = P0 + u1 (P1 - P0) + u2 (P2 - P1)
// and shared vertices first, the 4-D integrand becomes (xi, eta) with the
// singularity at xi = 0; for flat panels chi_P(u) - chi_Q(v) = xi D(eta) and
// the Jacobian carries xi^3, so the xi integral is exactly 1/3 and eta is
// integrated with an n^3 Gauss-Legendre rule.
#pragma once

#include "hm_internal.cuh"

namespace hm {

constexpr double INV_4PI = 0.079577471545947667884441881686257181;  // 1 / (4 pi)

// Panel record: x[0..6], y[7..13], z[14..20], area[21]; element k at p[k * stride].
__device__ __forceinline__ double regular_entry(const double *__restrict__ r, int rs, const double *__restrict__ c,
                                                int cs, const QuadParams &qp) {
    double cx[NQ], cy[NQ], cz[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        cx[q] = c[q * cs];
        cy[q] = c[(7 + q) * cs];
        cz[q] = c[(14 + q) * cs];
    }
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < NQ; ++p) {
        const double xp = r[p * rs], yp = r[(7 + p) * rs], zp = r[(14 + p) * rs];
        double sp = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double dx = xp - cx[q], dy = yp - cy[q], dz = zp - cz[q];
            sp = fma(qp.w[q], rsqrt(fma(dx, dx, fma(dy, dy, dz * dz))), sp);
        }
        s = fma(qp.w[p], sp, s);
    }
    return r[PT_AREA * rs] * c[PT_AREA * cs] * s * INV_4PI;
}

// Number of vertex indices shared by two triangles (0..3).
__device__ __forceinline__ int shared_vertices(const int32_t *a, const int32_t *b) {
    int k = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s)
        k += (a[s] == b[0]) | (a[s] == b[1]) | (a[s] == b[2]);
    return k;
}

// Orders the vertices of two touching triangles: shared ones first.  For a
// common edge the shared pair keeps its order in triangle a; for a common
// vertex each triangle is rotated cyclically to start at it.
__device__ __forceinline__ void touch_orient(const int32_t *a, const int32_t *b, int kind, int32_t P[3], int32_t Q[3]) {
    if (kind == 3) {
        for (int k = 0; k < 3; ++k) P[k] = Q[k] = a[k];
        return;
    }
    if (kind == 2) {
        int np = 0;
        for (int k = 0; k < 3; ++k) {
            const bool sh = (a[k] == b[0]) | (a[k] == b[1]) | (a[k] == b[2]);
            if (sh) { P[np] = Q[np] = a[k]; ++np; }
            else P[2] = a[k];
        }
        for (int k = 0; k < 3; ++k)
            if (b[k] != P[0] && b[k] != P[1]) Q[2] = b[k];
        return;
    }
    int ka = 0, kb = 0;
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y)
            if (a[x] == b[y]) { ka = x; kb = y; }
    for (int k = 0; k < 3; ++k) {
        P[k] = a[(ka + k) % 3];
        Q[k] = b[(kb + k) % 3];
    }
}

__device__ __forceinline__ int ss_regions(int kind) { return kind == 3 ? 6 : (kind == 2 ? 5 : 2); }

// Region r of the given kind at xi = 1: u, v in That and the eta-part of the
// Jacobian (the full Jacobian is xi^3 times this).
__device__ __forceinline__ void ss_region(int kind, int r, double e1, double e2, double e3, double &u0, double &u1,
                                          double &v0, double &v1, double &jac) {
    const double e12 = e1 * e2, e123 = e12 * e3;
    if (kind == 3) {
        jac = e1 * e12;
        switch (r) {
            case 0: u0 = 1.0; u1 = 1.0 - e1 + e12; v0 = 1.0 - e123; v1 = 1.0 - e1; break;
            case 1: u0 = 1.0 - e123; u1 = 1.0 - e1; v0 = 1.0; v1 = 1.0 - e1 + e12; break;
            case 2: u0 = 1.0; u1 = e1 - e12 + e123; v0 = 1.0 - e12; v1 = e1 - e12; break;
            case 3: u0 = 1.0 - e12; u1 = e1 - e12; v0 = 1.0; v1 = e1 - e12 + e123; break;
            case 4: u0 = 1.0 - e123; u1 = e1 - e123; v0 = 1.0; v1 = e1 - e12; break;
            default: u0 = 1.0; u1 = e1 - e12; v0 = 1.0 - e123; v1 = e1 - e123; break;
        }
    } else if (kind == 2) {
        jac = e1 * e12;
        switch (r) {
            case 0: jac = e1 * e1; u0 = 1.0; u1 = e1 * e3; v0 = 1.0 - e12; v1 = e1 - e12; break;
            case 1: u0 = 1.0; u1 = e1; v0 = 1.0 - e123; v1 = e12 - e123; break;
            case 2: u0 = 1.0 - e12; u1 = e1 - e12; v0 = 1.0; v1 = e123; break;
            case 3: u0 = 1.0 - e123; u1 = e12 - e123; v0 = 1.0; v1 = e1; break;
            default: u0 = 1.0 - e123; u1 = e1 - e123; v0 = 1.0; v1 = e12; break;
        }
    } else {
        jac = e2;
        if (r == 0) { u0 = 1.0; u1 = e1; v0 = e2; v1 = e2 * e3; }
        else { u0 = e2; u1 = e2 * e3; v0 = 1.0; v1 = e1; }
    }
}

// Edge vectors of an ordered pair: a1 = P1 - P0, a2 = P2 - P1, b1 = Q1 - Q0, b2 = Q2 - Q1.
struct PairGeom {
    double a1[3], a2[3], b1[3], b2[3];
};

__device__ __forceinline__ PairGeom pair_geom(const double *V, const int32_t P[3], const int32_t Q[3]) {
    PairGeom g;
    for (int d = 0; d < 3; ++d) {
        const double p0 = V[3 * (int64_t)P[0] + d], p1 = V[3 * (int64_t)P[1] + d], p2 = V[3 * (int64_t)P[2] + d];
        const double q0 = V[3 * (int64_t)Q[0] + d], q1 = V[3 * (int64_t)Q[1] + d], q2 = V[3 * (int64_t)Q[2] + d];
        g.a1[d] = p1 - p0;
        g.a2[d] = p2 - p1;
        g.b1[d] = q1 - q0;
        g.b2[d] = q2 - q1;
    }
    return g;
}

// One point of the regularised rule: w * jac / |D| with
// D = (u0 a1 + u1 a2) - (v0 b1 + v1 b2).
__device__ __forceinline__ double ss_point(const PairGeom &g, int kind, int r, int k1, int k2, int k3,
                                           const QuadParams &qp) {
    double u0, u1, v0, v1, jac;
    ss_region(kind, r, qp.gx[k1], qp.gx[k2], qp.gx[k3], u0, u1, v0, v1, jac);
    double dd = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double D = (u0 * g.a1[d] + u1 * g.a2[d]) - (v0 * g.b1[d] + v1 * g.b2[d]);
        dd = fma(D, D, dd);
    }
    return qp.gw[k1] * qp.gw[k2] * qp.gw[k3] * jac * rsqrt(dd);
}

// Whole touching-pair entry by one thread (used where touching pairs are rare).
__device__ __noinline__ static double singular_entry_serial(const double *V, const int32_t *ta, const int32_t *tb, int kind, double area_a,
                                        double area_b, const QuadParams &qp) {
    int32_t P[3], Q[3];
    touch_orient(ta, tb, kind, P, Q);
    const PairGeom g = pair_geom(V, P, Q);
    const int n = qp.ss_n, R = ss_regions(kind);
    double s = 0.0;
    for (int r = 0; r < R; ++r)
        for (int k1 = 0; k1 < n; ++k1)
            for (int k2 = 0; k2 < n; ++k2)
                for (int k3 = 0; k3 < n; ++k3) s += ss_point(g, kind, r, k1, k2, k3, qp);
    // 4 |Ti| |Tj| from the two parametrisations, 1/3 from the xi integral
    return 4.0 * area_a * area_b * (s / 3.0) * INV_4PI;
}

}  // namespace hm
