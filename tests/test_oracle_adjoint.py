"""Pins of the oracle's differentiation pieces (CPU).

* potential_matrix: on the unit sphere the exact density of an exterior
  point source p has, outside the sphere, the Kelvin image field
  U_ext(x) = 1 / (4 pi | |p| x - p/|p| |); E applied to that density sampled
  at the centroids must approach U_ext at the evaluation points as the mesh
  is refined (geometry + P0 error, O(h^2)).
* misfit_loss_and_gradients: the adjoint gradients against central finite
  differences of the loss itself (which only needs forward solves), at a
  base point c != 1 so that A diag(c) is not symmetric.
"""
import math

import numpy as np

import meshgen


def _exterior_field(x, p):
    p = np.asarray(p, dtype=np.float64)
    pn = np.linalg.norm(p)
    return 1.0 / (4.0 * math.pi * np.linalg.norm(pn * x - p[None, :] / pn, axis=1))


def test_potential_matrix_reproduces_exterior_field(orc):
    p = np.array([3.0, 0.0, 0.0])
    pts = meshgen.exterior_points(7, 64, 2.5)
    exact = _exterior_field(pts, p)
    errs = []
    for L in (2, 3, 4):
        V, T = meshgen.icosphere(L)
        cent = V[T].mean(axis=1)
        u = orc.point_source_density(cent, p)
        E = orc.potential_matrix(V, T, pts)
        errs.append(np.abs(E @ u - exact).max() / np.abs(exact).max())
    rates = [e1 / e2 for e1, e2 in zip(errs, errs[1:])]
    assert min(rates) > 3.0, (errs, rates)
    assert errs[-1] < 2e-3, errs


def test_potential_matrix_rows_are_the_potential(orc):
    V, T = meshgen.icosphere(2)
    pts = meshgen.exterior_points(3, 8, 2.5)
    E = orc.potential_matrix(V, T, pts)
    a = np.random.default_rng(0).standard_normal(T.shape[0])
    assert np.abs(E @ a - orc.potential(V, T, a, pts)).max() <= 1e-14 * np.abs(E).sum(axis=1).max()


def _problem(orc, L=2, npts=64):
    V, T = meshgen.icosphere(L)
    pts = meshgen.exterior_points(11, npts, 2.5)
    A = orc.dense_matrix(V, T)
    E = orc.potential_matrix(V, T, pts)
    f = orc.load_vector(V, T, [3.0, 0.0, 0.0])[0]
    target = orc.point_source_potential(pts, [0.0, 0.0, 3.0])
    return A, E, f, target


def test_misfit_gradients_match_central_differences(orc):
    A, E, f, target = _problem(orc)
    n = f.shape[0]
    rng = np.random.default_rng(5)
    c = 1.0 + 0.2 * rng.uniform(-1.0, 1.0, n)
    L0, alpha, gf, gc = orc.misfit_loss_and_gradients(A, E, f, c, target)

    def loss(ff, cc):
        return orc.misfit_loss_and_gradients(A, E, ff, cc, target)[0]

    for _ in range(4):
        d = rng.standard_normal(n)
        # L is quadratic in f: central differences are exact up to rounding
        h = 1e-2 * np.linalg.norm(f) / np.linalg.norm(d)
        fd = (loss(f + h * d, c) - loss(f - h * d, c)) / (2 * h)
        assert abs(fd - gf @ d) <= 1e-7 * abs(gf @ d) + 1e-12 * L0, (fd, gf @ d)
        h = 1e-5
        fd = (loss(f, c + h * d) - loss(f, c - h * d)) / (2 * h)
        assert abs(fd - gc @ d) <= 1e-6 * abs(gc @ d) + 1e-10 * L0, (fd, gc @ d)


def test_misfit_c_gradient_is_a_reparametrisation(orc):
    """Scaling column j by c_j and the density by 1/c_j leaves the product
    unchanged, so dL/dc_j = -alpha_j (dL/dalpha)_j / c_j."""
    A, E, f, target = _problem(orc)
    c = 1.0 + 0.1 * np.random.default_rng(2).uniform(-1.0, 1.0, f.shape[0])
    L0, alpha, gf, gc = orc.misfit_loss_and_gradients(A, E, f, c, target)
    g_alpha = (2.0 / E.shape[0]) * (E.T @ (E @ alpha - target))
    assert np.linalg.norm(gc + alpha * g_alpha / c) <= 1e-9 * np.linalg.norm(gc)
