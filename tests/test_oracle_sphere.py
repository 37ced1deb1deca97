"""Analytic pins of the whole oracle discretisation on the unit sphere.

On |x| = 1 the single-layer operator (Example 2.1) satisfies S 1 = 1 and
S Y_lm = Y_lm / (2l+1); the exterior point source p gives the density
u = (1 - t^2) / (4 pi |p| (1 - 2 t cos g + t^2)^(3/2)), t = 1/|p|, and the
interior potential 1/(4 pi |x - p|) (the eps(h) check of Sec. 4.3).  Flat
triangles carry an O(h^2) geometry error, so the checks are on decay with
the level rather than on a fixed constant.
"""
import math

import numpy as np
import pytest

import meshgen


@pytest.fixture(scope="module")
def ladder(orc):
    out = {}
    for L in (1, 2, 3, 4):
        V, T = meshgen.icosphere(L)
        A = orc.dense_matrix(V, T)
        c, a = orc.panel_geometry(V, T)
        out[L] = (V, T, A, c, a)
    return out


def test_dense_matrix_spd(ladder):
    V, T, A, c, a = ladder[3]
    assert np.abs(A - A.T).max() < 1e-10 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_constant_density_gives_one(orc, ladder):
    errs, rows = [], []
    for L, (V, T, A, c, a) in sorted(ladder.items()):
        alpha = orc.lu_solve(A, a)  # S alpha = 1 tested with phi_i
        errs.append(np.abs(alpha - 1).max())
        rows.append(np.abs(A.sum(1) / a - 1).max())  # S 1 ~ 1 row-wise
    assert all(e2 < 0.6 * e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 6e-3
    assert all(r2 < r1 for r1, r2 in zip(rows, rows[1:])) and rows[-1] < 1e-2


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4, 6])
def test_spherical_harmonic_eigenvalues(orc, ladder, l):
    errs = []
    for L, (V, T, A, c, a) in sorted(ladder.items()):
        if L < 2:
            continue
        Y = meshgen.real_sph_harm(l, min(l, 1), c)
        rq = (Y @ A @ Y) / np.sum(a * Y * Y)
        errs.append(abs(rq * (2 * l + 1) - 1))
    assert all(e2 < 0.5 * e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.03


def test_point_source_density_and_potential(orc, ladder):
    p = np.array([3.0, 0.0, 0.0])
    pts = meshgen.interior_points(1806, 64)
    Uex = orc.point_source_potential(pts, p)
    dens, pot = [], []
    for L, (V, T, A, c, a) in sorted(ladder.items()):
        f = orc.load_vector(V, T, p)[0]
        alpha = orc.lu_solve(A, f)
        u = orc.point_source_density(c, p)
        dens.append(np.abs(alpha - u).max() / np.abs(u).max())
        pot.append(np.abs(orc.potential(V, T, alpha, pts) - Uex).max())
    assert all(e2 < 0.7 * e1 for e1, e2 in zip(dens, dens[1:])), dens
    # eps(h) decays about like N^-1.5 (factor 8 per level) on the sphere
    assert all(e2 < 0.2 * e1 for e1, e2 in zip(pot, pot[1:])), pot
    assert pot[-1] < 1e-7


def test_load_vector_closed_form_far_source(orc):
    # for a distant source the load vector tends to |T_i| / (4 pi |c_i - p|)
    V, T = meshgen.icosphere(2)
    c, a = orc.panel_geometry(V, T)
    p = np.array([40.0, -10.0, 5.0])
    f = orc.load_vector(V, T, p)[0]
    approx = a / (4 * math.pi * np.linalg.norm(c - p, axis=1))
    assert np.abs(f / approx - 1).max() < 1e-5


def test_potential_of_constant_density(orc, ladder):
    # S~ 1 = 1 inside the unit sphere (Eq. 2 with u = 1)
    V, T, A, c, a = ladder[4]
    pts = meshgen.interior_points(3, 16)
    val = orc.potential(V, T, np.ones(T.shape[0]), pts)
    assert np.abs(val - 1).max() < 3e-3
