"""Pins of the oracle's quadrature rules (Sec. 4.1 'higher-order quadrature')."""
import math
import os

import numpy as np
import pytest

from oracle.quadrature import gauss_legendre01, tri7

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tri7_dunavant_degree5.txt")


def _tri_integral(a, b):
    # int over {x, y >= 0, x + y <= 1} of x^a y^b = a! b! / (a + b + 2)!
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


def test_tri7_matches_published_table():
    bary, w = tri7()
    tab = np.loadtxt(GOLDEN)
    # expand orbits of the table
    pts, wts = [], []
    for wt, b1, b2, b3 in tab:
        orbit = {(b1, b2, b3), (b2, b3, b1), (b3, b1, b2)}
        for o in sorted(orbit):
            pts.append(o)
            wts.append(wt)
    pts, wts = np.array(pts), np.array(wts)
    for p, wt in zip(bary, w):
        k = np.argmin(np.abs(pts - p).sum(1))
        assert np.abs(pts[k] - p).max() < 1e-14
        assert abs(wts[k] - wt) < 1e-14
    assert abs(w.sum() - 1.0) < 1e-15


def test_tri7_exact_to_degree5_not_6():
    bary, w = tri7()
    x, y = bary[:, 1], bary[:, 2]
    for deg in range(6):
        for a in range(deg + 1):
            b = deg - a
            q = 0.5 * np.sum(w * x ** a * y ** b)
            assert abs(q - _tri_integral(a, b)) < 1e-15 * 10, (a, b)
    errs = [abs(0.5 * np.sum(w * x ** a * y ** (6 - a)) - _tri_integral(a, 6 - a)) for a in range(7)]
    assert max(errs) > 1e-6


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_gauss_legendre_exactness(n):
    x, w = gauss_legendre01(n)
    assert ((x > 0) & (x < 1)).all()
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
    if n <= 5:
        assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


def test_gauss_legendre_two_point_nodes():
    x, w = gauss_legendre01(2)
    assert np.allclose(np.sort(x), [0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6], atol=1e-15)
    assert np.allclose(w, 0.5, atol=1e-15)
