"""Input generators: topology and geometry of the generated meshes."""
import math

import numpy as np
import pytest

import meshgen


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_icosphere_counts_and_manifold(level):
    V, T = meshgen.icosphere(level)
    assert T.shape == (20 * 4 ** level, 3) and T.dtype == np.int32
    assert V.shape == (10 * 4 ** level + 2, 3)
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-15)
    # closed 2-manifold: every undirected edge in exactly two faces, opposite directions
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]]).astype(np.int64)
    fwd = set(map(tuple, e))
    assert len(fwd) == e.shape[0]
    assert all((b, a) in fwd for a, b in fwd)
    # Euler characteristic of the sphere
    assert V.shape[0] - e.shape[0] // 2 + T.shape[0] == 2
    # outward orientation
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    assert ((n * V[T].mean(1)).sum(1) > 0).all()


def test_icosphere_deterministic():
    a = meshgen.icosphere(3)
    b = meshgen.icosphere(3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_real_sph_harm_orthonormal():
    # product Gauss-Legendre (cos theta) x trapezoid (phi), exact for l <= 4 products
    x, w = np.polynomial.legendre.leggauss(20)
    ph = np.linspace(0, 2 * math.pi, 41)[:-1]
    ct, pp = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    xyz = np.stack([st * np.cos(pp), st * np.sin(pp), ct], -1)
    W = np.outer(w, np.full(ph.size, 2 * math.pi / ph.size))
    modes = [(l, m) for l in range(5) for m in range(-l, l + 1)]
    Y = np.stack([meshgen.real_sph_harm(l, m, xyz) for l, m in modes])
    G = np.einsum("aij,bij,ij->ab", Y, Y, W)
    assert np.allclose(G, np.eye(len(modes)), atol=1e-12)
    # Y_00 = 1/sqrt(4 pi), Y_10 = sqrt(3/(4 pi)) z
    assert np.allclose(Y[0], 1 / math.sqrt(4 * math.pi))
    assert np.allclose(Y[2], math.sqrt(3 / (4 * math.pi)) * ct)


def test_bump_sphere_radius_and_seed():
    V, T, modes = meshgen.bump_sphere(3, 1808)
    r = np.linalg.norm(V, axis=1)
    assert r.min() >= 0.5 and len(modes) == 8 and len({(l, m) for l, m, _ in modes}) == 8
    assert all(l <= 4 for l, _, _ in modes)
    V2, _, modes2 = meshgen.bump_sphere(3, 1808)
    assert np.array_equal(V, V2) and modes == modes2


def test_point_sources_outside_stretched():
    s = np.array([2.0, 0.5, 1.0])
    p = meshgen.point_sources(11, 64, scales=s)
    rr = np.linalg.norm(p, axis=1)
    assert ((rr >= 2) & (rr <= 4)).all()
    assert (((p / s) ** 2).sum(1) > 1.1 ** 2).all()


def test_interior_and_exterior_points():
    q = meshgen.interior_points(3, 200)
    assert (np.linalg.norm(q, axis=1) <= 0.5).all()
    e = meshgen.exterior_points(3, 100, 2.5)
    assert np.allclose(np.linalg.norm(e, axis=1), 2.5)
