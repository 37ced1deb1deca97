"""Pins of the oracle's Galerkin entries (Eq. 4, Sec. 4.1 quadrature).

The regularised touching-pair integrals are checked against things fixed by
the mathematics, not by the oracle: exact tiling of That x That by the
regions, exponential self-convergence in the Gauss order, and an independent
evaluation (closed-form potential of a uniform flat triangle for the inner
integral, double-exponential quadrature for the outer one).
"""
import itertools
import math

import numpy as np
import pytest

import meshgen


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


@pytest.mark.parametrize("kind", [3, 2, 1])
def test_regions_tile_reference_square(orc, kind):
    x, w = _gl(7)
    XI, E1, E2, E3 = (a.ravel() for a in np.meshgrid(x, x, x, x, indexing="ij"))
    W = np.einsum("i,j,k,l->ijkl", w, w, w, w).ravel()
    u, v, jac = orc.ss_points(kind, XI, E1, E2, E3)
    # all points inside That = {0 <= u2 <= u1 <= 1}
    for z in (u, v):
        assert (z[..., 1] >= -1e-15).all() and (z[..., 1] <= z[..., 0] + 1e-15).all() and (z[..., 0] <= 1 + 1e-15).all()
    tri = lambda a, b: 1.0 / ((b + 1) * (a + b + 2))
    for a, b, c, d in itertools.product(range(3), repeat=4):
        got = np.sum(W[None] * jac * u[..., 0] ** a * u[..., 1] ** b * v[..., 0] ** c * v[..., 1] ** d)
        assert abs(got - tri(a, b) * tri(c, d)) < 1e-14, (a, b, c, d)


def _touching_pairs(T):
    """one (i, j) per kind: coincident, common edge, common vertex"""
    out = {3: (0, 0)}
    s0 = set(T[0])
    for j in range(1, T.shape[0]):
        k = len(s0 & set(T[j]))
        if k in (1, 2) and k not in out:
            out[k] = (0, j)
    return out


def _tri_pot(X, P):
    """int_P 1/|x - y| dsigma_y for a flat triangle P (closed form), X [k,3]."""
    A, B, C = P
    nrm = np.cross(B - A, C - A)
    nrm /= np.linalg.norm(nrm)
    h = (X - A) @ nrm
    ah = np.abs(h)
    Xp = X - h[:, None] * nrm
    tot = np.zeros(X.shape[0])
    for P0, P1 in ((A, B), (B, C), (C, A)):
        L = np.linalg.norm(P1 - P0)
        t = (P1 - P0) / L
        m = np.cross(t, nrm)
        d = (P0 - Xp) @ m
        sm = (P0 - Xp) @ t
        sp = (P1 - Xp) @ t
        Rm = np.linalg.norm(X - P0, axis=1)
        Rp = np.linalg.norm(X - P1, axis=1)
        R0 = d * d + h * h
        # s + R without cancellation for s < 0: (R + s)(R - s) = R0
        with np.errstate(divide="ignore", invalid="ignore"):
            ap = np.where(sp >= 0, sp + Rp, R0 / (Rp - sp))
            am = np.where(sm >= 0, sm + Rm, R0 / (Rm - sm))
            lg = np.where(np.abs(d) > 0, d * np.log(ap / am), 0.0)
            at = np.arctan(d * sp / (R0 + ah * Rp)) - np.arctan(d * sm / (R0 + ah * Rm))
        tot += lg - ah * np.where(np.abs(d) > 0, at, 0.0)
    return tot


def _tanh_sinh(h=0.1, kmax=40):
    t = np.arange(-kmax, kmax + 1) * h
    s = 0.5 * math.pi * np.sinh(t)
    x = 0.5 * (1 + np.tanh(s))
    w = h * 0.25 * math.pi * np.cosh(t) / np.cosh(s) ** 2
    keep = (x > 0) & (x < 1) & (w > 0)
    return x[keep], w[keep]


def _independent_entry(P, Q):
    """int_P int_Q G by closed-form inner integral and tanh-sinh outer rule on
    the collapsed square x = A + u (B - A) + u v (C - B)."""
    A, B, C = P
    x, w = _tanh_sinh()
    U, Vv = np.meshgrid(x, x, indexing="ij")
    Wt = np.outer(w, w)
    X = A + U.ravel()[:, None] * (B - A) + (U * Vv).ravel()[:, None] * (C - B)
    jac = np.linalg.norm(np.cross(B - A, C - A)) * U.ravel()
    return np.sum(Wt.ravel() * jac * _tri_pot(X, Q)) / (4 * math.pi)


def test_closed_form_triangle_potential_against_brute_force():
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.8, 0.0]])
    X = np.array([[0.5, 0.4, 0.7], [-0.3, 1.2, -0.2], [2.0, 0.1, 0.05]])
    # brute force: 7-point rule on a 4^6 subdivision of P
    tris = [P]
    for _ in range(6):
        nt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nt += [np.array(t) for t in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))]
        tris = nt
    from oracle.quadrature import tri7
    bary, w7 = tri7()
    tris = np.array(tris)
    pts = np.einsum("qk,tkd->tqd", bary, tris).reshape(-1, 3)
    ar = 0.5 * np.linalg.norm(np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]), axis=1)
    wt = (ar[:, None] * w7[None]).ravel()
    for x in X:
        bf = np.sum(wt / np.linalg.norm(pts - x, axis=1))
        assert abs(_tri_pot(x[None], P)[0] - bf) < 1e-10 * abs(bf)


@pytest.mark.parametrize("mesh", ["sphere", "bumped"])
def test_singular_entries_self_convergence_and_independent_value(orc, mesh):
    if mesh == "sphere":
        V, T = meshgen.icosphere(2)
    else:
        V, T, _ = meshgen.bump_sphere(2, 1808)
    pairs = _touching_pairs(T)
    for kind, (i, j) in pairs.items():
        assert orc.touch(T, i, j) == kind
        vals = {n: orc.entry(V, T, i, j, orc.Quad(n)) for n in (4, 6, 8, 10, 12, 16)}
        ref = vals[16]
        errs = [abs(vals[n] - ref) / ref for n in (4, 6, 8, 10)]
        assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
        assert errs[-1] < 1e-10 and abs(vals[12] - ref) / ref < 1e-12
        # independent evaluation
        P = V[T[i]]
        Q = V[T[j]]
        ind = _independent_entry(P, Q)
        assert abs(ind - ref) / ref < 1e-12, (kind, ind, ref)


def test_singular_entries_symmetric(orc):
    V, T, _ = meshgen.bump_sphere(2, 1808)
    q = orc.Quad(16)
    for kind, (i, j) in _touching_pairs(T).items():
        a, b = orc.entry(V, T, i, j, q), orc.entry(V, T, j, i, q)
        assert abs(a - b) / abs(a) < 1e-13


def test_regular_rule_error_decays_like_degree_5(orc):
    """A non-touching pair at growing separation d: the 7x7 rule approaches
    the exact integral with error O((h/d)^6); a wrong point or weight in the
    rule drops the order and fails the rate check."""
    P = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.03, 0.08, 0.0]])
    shift = np.array([0.6, 0.3, 1.0])
    shift /= np.linalg.norm(shift)
    errs = []
    for d in (0.2, 0.4, 0.8, 1.6):
        Q = P[[0, 2, 1]] + d * shift
        V = np.concatenate([P, Q])
        T = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
        a = orc.entry(V, T, 0, 1)
        exact = _independent_entry(P, Q)
        errs.append(abs(a - exact) / exact)
    rates = [math.log2(e1 / e2) for e1, e2 in zip(errs, errs[1:])]
    assert min(rates) > 5.0, (errs, rates)
    assert errs[-1] < 1e-10


def test_far_entry_tends_to_point_interaction(orc):
    V, T = meshgen.icosphere(3)
    c, a = orc.panel_geometry(V, T)
    i = 0
    j = int(np.argmax(np.linalg.norm(c - c[0], axis=1)))
    approx = a[i] * a[j] / (4 * math.pi * np.linalg.norm(c[i] - c[j]))
    assert abs(orc.entry(V, T, i, j) - approx) / approx < 2e-3
