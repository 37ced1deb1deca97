"""Quadrature rules of the oracle (test infrastructure only).

* ``tri7``: the degree-5, 7-point rule on a triangle (Radon's rule; Stroud
  T2:5-1, Dunavant degree 5).  The paper (Sec. 4.1) only asks for
  "higher-order quadrature"; the 7-point rule on far panels is the reading
  taken here.  Points are barycentric, weights sum to one.
* ``gauss_legendre01``: n-point Gauss-Legendre on [0, 1], from the library
  routine numpy.polynomial.legendre.leggauss.
"""
from __future__ import annotations

import math

import numpy as np


def tri7():
    """Barycentric points (7,3) and weights (7,), weights summing to 1."""
    s15 = math.sqrt(15.0)
    a1 = (6.0 - s15) / 21.0
    a2 = (6.0 + s15) / 21.0
    w1 = (155.0 - s15) / 1200.0
    w2 = (155.0 + s15) / 1200.0
    third = 1.0 / 3.0
    bary = np.array([
        [third, third, third],
        [a1, a1, 1.0 - 2.0 * a1],
        [a1, 1.0 - 2.0 * a1, a1],
        [1.0 - 2.0 * a1, a1, a1],
        [a2, a2, 1.0 - 2.0 * a2],
        [a2, 1.0 - 2.0 * a2, a2],
        [1.0 - 2.0 * a2, a2, a2],
    ], dtype=np.float64)
    w = np.array([9.0 / 40.0, w1, w1, w1, w2, w2, w2], dtype=np.float64)
    return bary, w


def gauss_legendre01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w
