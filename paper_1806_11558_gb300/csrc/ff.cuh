// ff.cuh -- double-float ("float-float") arithmetic for far-field kernel
// evaluations.
//
// On GB300 the FP64 pipe issues 2 DFMA per SM per clock against 128 FFMA, so
// the batched ACA (Sec. 2.3), whose entries are far-field (admissible blocks,
// well-separated panels), evaluates the 7x7 quadrature sum with pairs of
// floats carrying about 48 significant bits:
//   * Knuth's TwoSum and the FMA-based TwoProduct (Dekker's exact product)
//     give the rounding errors of a + b and a * b exactly;
//   * the reciprocal square root starts from the hardware estimate rsqrtf and
//     takes one Newton-Raphson step whose residual 1 - r y0^2 is formed from
//     exact products, so the result is accurate to ~1e-13 relative;
//   * sums of positive terms carry their low parts separately and are
//     normalised once at the end.
// Differences of points are taken relative to the panel centroids, so the
// representation error of a coordinate is relative to the panel size, not to
// the distance from the origin; that also holds for neighbouring panels, so
// the regular near-field entries (non-touching pairs of dense leaves) use the
// same evaluation.
#pragma once

#include "hm_internal.cuh"

namespace hm {

// s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e == a + b exactly, valid when |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// p + e == a * b exactly
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// (h, l) of a double: h = nearest float, l = nearest float of the remainder
__device__ __forceinline__ void split_double(double x, float &h, float &l) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

// Float panel record of the far-field evaluation (rows of the float panel
// table PF, component-major like the FP64 one):
//   [0, 21)  a_hi : offsets x_q - c of the 7 quadrature points (x: 0..6, y: 7..13, z: 14..20)
//   [21, 42) a_lo
//   [42, 45) c_hi : centroid;  [45, 48) c_lo
//   [48] wa_hi, [49] wa_lo : |T| / sqrt(4 pi)
//   [50, 53) vertex indices (int bits)
constexpr int PF_ROWS = 53;
constexpr int PF_AH = 0, PF_AL = 21, PF_CH = 42, PF_CL = 45, PF_WA = 48, PF_VID = 50;
// sqrt(4 pi)
constexpr double SQRT_4PI = 3.5449077018110320545963349666822903655950989122447742564276155;

// A float pair h + l (|l| <= ulp(h) / 2 when normalised).
struct __align__(8) FF {
    float h, l;
};

__device__ __forceinline__ FF ff_from(double x) {
    FF r;
    split_double(x, r.h, r.l);
    return r;
}
__device__ __forceinline__ double ff_to(FF a) { return (double)a.h + (double)a.l; }

// a * b, normalised, to ~2^-47 relative
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    float ph, pe;
    two_prod(a.h, b.h, ph, pe);
    pe = __fmaf_rn(a.h, b.l, pe);
    pe = __fmaf_rn(a.l, b.h, pe);
    FF r;
    fast_two_sum(ph, pe, r.h, r.l);
    return r;
}

// (hs, lo) -= b * c: the high parts subtract exactly (TwoSum) and every
// rounding error goes to lo, so a chain of these followed by one
// fast_two_sum(hs, lo) is accurate to ~2^-48 of the largest term
__device__ __forceinline__ void ff_sub_prod(float &hs, float &lo, FF b, FF c) {
    float ph, pe;
    two_prod(b.h, c.h, ph, pe);
    pe = __fmaf_rn(b.h, c.l, pe);
    pe = __fmaf_rn(b.l, c.h, pe);
    float s, e;
    two_sum(hs, -ph, s, e);
    hs = s;
    lo = __fadd_rn(lo, __fsub_rn(e, pe));
}

// Regular entry a_ij = |Ti||Tj|/(4 pi) sum_p sum_q w_p w_q / |x_p - y_q| for
// panel records R (row, test) and C (column, trial); element k of a record at
// R[k * rs].  wq_h / wq_l: the 7 weights as float pairs.  Returns the float
// pair (eh, el), not normalised.
__device__ __forceinline__ void regular_entry_ff2(const float *__restrict__ R, int rs, const float *__restrict__ C,
                                                  int cs, const float *wq_h, const float *wq_l, float &eh_out,
                                                  float &el_out) {
    // D = c_R - c_C in float-float, to 2^-48 |D|: the hi and lo differences
    // are both exact (TwoSum), and only their combination rounds, so
    // neighbouring panels (|D| ~ panel size) keep full relative accuracy
    float Dh[3], Dl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float s, e, t, f, u, g;
        two_sum(R[(PF_CH + d) * rs], -C[(PF_CH + d) * cs], s, e);
        two_sum(R[(PF_CL + d) * rs], -C[(PF_CL + d) * cs], t, f);
        two_sum(e, t, u, g);
        float sh, sl;
        two_sum(s, u, sh, sl);
        fast_two_sum(sh, __fadd_rn(sl, __fadd_rn(g, f)), Dh[d], Dl[d]);
    }
    // column offsets b_q (hi, lo)
    float bh[3][NQ], bl[3][NQ];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            bh[d][q] = C[(PF_AH + 7 * d + q) * cs];
            bl[d][q] = C[(PF_AL + 7 * d + q) * cs];
        }
    float acc_h = 0.0f, acc_l = 0.0f;
    // the outer loop stays rolled: the 7-fold inner body is ~500 instructions
    // and one copy of it keeps the instruction cache warm
#pragma unroll 1
    for (int p = 0; p < NQ; ++p) {
        // X_p = D + a_p
        float Xh[3], Xl[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float s, e;
            two_sum(Dh[d], R[(PF_AH + 7 * d + p) * rs], s, e);
            e = __fadd_rn(e, __fadd_rn(Dl[d], R[(PF_AL + 7 * d + p) * rs]));
            fast_two_sum(s, e, Xh[d], Xl[d]);
        }
        float sp_h = 0.0f, sp_l = 0.0f;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            // r^2 = |X_p - b_q|^2
            float ph[3], pl[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float s, e;
                two_sum(Xh[d], -bh[d][q], s, e);
                e = __fadd_rn(e, __fsub_rn(Xl[d], bl[d][q]));
                two_prod(s, s, ph[d], pl[d]);
                pl[d] = __fmaf_rn(__fmul_rn(2.0f, s), e, pl[d]);
            }
            float t1, u1, t2, u2;
            two_sum(ph[0], ph[1], t1, u1);
            two_sum(t1, ph[2], t2, u2);
            const float r2l = __fadd_rn(__fadd_rn(__fadd_rn(pl[0], pl[1]), __fadd_rn(pl[2], u1)), u2);
            // 1 / sqrt(r2): estimate + one Newton step with an exact residual
            const float y0 = rsqrtf(t2);
            float yh, yl;
            two_prod(y0, y0, yh, yl);
            float mh, ml;
            two_prod(t2, yh, mh, ml);
            ml = __fmaf_rn(t2, yl, ml);
            ml = __fmaf_rn(r2l, yh, ml);
            const float del = __fsub_rn(__fsub_rn(1.0f, mh), ml);
            const float corr = __fmul_rn(__fmul_rn(0.5f, y0), del);
            // sp += w_q (y0 + corr)
            float qh, ql;
            two_prod(wq_h[q], y0, qh, ql);
            ql = __fmaf_rn(wq_h[q], corr, ql);
            ql = __fmaf_rn(wq_l[q], y0, ql);
            float s, e;
            two_sum(sp_h, qh, s, e);
            sp_h = s;
            sp_l = __fadd_rn(sp_l, __fadd_rn(e, ql));
        }
        // acc += w_p sp
        float sh, sl;
        fast_two_sum(sp_h, sp_l, sh, sl);
        float qh, ql;
        two_prod(wq_h[p], sh, qh, ql);
        ql = __fmaf_rn(wq_h[p], sl, ql);
        ql = __fmaf_rn(wq_l[p], sh, ql);
        float s, e;
        two_sum(acc_h, qh, s, e);
        acc_h = s;
        acc_l = __fadd_rn(acc_l, __fadd_rn(e, ql));
    }
    // times (|T_R| / sqrt(4 pi)) (|T_C| / sqrt(4 pi)), then to double
    float ah, al;
    fast_two_sum(acc_h, acc_l, ah, al);
    float wh, wl;
    two_prod(R[PF_WA * rs], C[PF_WA * cs], wh, wl);
    wl = __fmaf_rn(R[PF_WA * rs], C[(PF_WA + 1) * cs], wl);
    wl = __fmaf_rn(R[(PF_WA + 1) * rs], C[PF_WA * cs], wl);
    float eh, el;
    two_prod(ah, wh, eh, el);
    el = __fmaf_rn(ah, wl, el);
    el = __fmaf_rn(al, wh, el);
    eh_out = eh;
    el_out = el;
}

__device__ __forceinline__ double regular_entry_ff(const float *__restrict__ R, int rs, const float *__restrict__ C,
                                                   int cs, const float *wq_h, const float *wq_l) {
    float eh, el;
    regular_entry_ff2(R, rs, C, cs, wq_h, wq_l, eh, el);
    return (double)eh + (double)el;
}

}  // namespace hm
