"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only generates inputs: triangle meshes of (bumped / stretched)
spheres, point-source locations and evaluation points.  It holds none of the
method's arithmetic (no quadrature, no kernel evaluation, no clustering), so
that both sides of every parity test start from byte-identical inputs while
sharing no computation.

The paper's own geometries (unit cube, gearwheel; Sec. 4.3) are parametric
quadrangular meshes that are not available; flat-triangle icospheres stand in
for them.  The single-layer operator on the unit sphere has closed-form
eigenvalues, which is what makes the sphere useful for pinning the oracle.
"""
from __future__ import annotations

import math

import numpy as np

MASTER_SEED = 1806

__all__ = [
    "MASTER_SEED", "icosphere", "bump_sphere", "stretch", "real_sph_harm",
    "point_sources", "exterior_points", "interior_points", "config",
]


def _icosahedron():
    """The 12 vertices (cyclic permutations of (0, ±1, ±φ), normalised) and
    20 faces of the regular icosahedron, each face oriented counter-clockwise
    seen from outside."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((0.0, s1, s2 * phi))
            v.append((s1, s2 * phi, 0.0))
            v.append((s2 * phi, 0.0, s1))
    V = np.array(v, dtype=np.float64)
    V /= np.linalg.norm(V, axis=1)[:, None]
    # faces = triples of mutually adjacent vertices (edge length 2 before normalising)
    d2 = ((V[:, None, :] - V[None, :, :]) ** 2).sum(-1)
    edge = np.isclose(d2, d2[d2 > 1e-12].min())
    faces = []
    for a in range(12):
        for b in range(a + 1, 12):
            if not edge[a, b]:
                continue
            for c in range(b + 1, 12):
                if edge[a, c] and edge[b, c]:
                    faces.append((a, b, c))
    F = np.array(faces, dtype=np.int64)
    assert F.shape == (20, 3)
    # orient outward
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = (n * V[F].mean(axis=1)).sum(1) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def icosphere(level: int):
    """Icosphere of the given subdivision level.

    Each refinement splits every triangle into four through its edge
    midpoints (shared between neighbours) and pushes the new vertices onto
    the unit sphere.  Returns (V float64 [nv,3], T int32 [N,3]) with
    N = 20*4**level and nv = 10*4**level + 2; faces are counter-clockwise
    seen from outside.  The ordering is fixed by this generator.
    """
    if level < 0:
        raise ValueError("level must be >= 0")
    V, F = _icosahedron()
    for _ in range(level):
        nv = V.shape[0]
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
        key = np.sort(e, axis=1)
        uniq, inv = np.unique(key[:, 0] * nv + key[:, 1], return_inverse=True)
        a, b = uniq // nv, uniq % nv
        mid = V[a] + V[b]
        mid /= np.linalg.norm(mid, axis=1)[:, None]
        nf = F.shape[0]
        m01 = nv + inv[:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:]
        c0, c1, c2 = F[:, 0], F[:, 1], F[:, 2]
        Fn = np.stack([
            np.stack([c0, m01, m20], 1),
            np.stack([m01, c1, m12], 1),
            np.stack([m20, m12, c2], 1),
            np.stack([m01, m12, m20], 1),
        ], axis=1).reshape(-1, 3)
        V = np.concatenate([V, mid])
        F = Fn
    return np.ascontiguousarray(V), np.ascontiguousarray(F.astype(np.int32))


def _assoc_legendre(l: int, m: int, x):
    """P_l^m(x) without the Condon-Shortley phase, m >= 0 (three-term recurrence)."""
    x = np.asarray(x, dtype=np.float64)
    pmm = np.ones_like(x)
    if m > 0:
        s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
        fact = 1.0
        for _ in range(m):
            pmm = pmm * fact * s
            fact += 2.0
    if l == m:
        return pmm
    pm1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pm1
    p2, p1 = pmm, pm1
    for ll in range(m + 2, l + 1):
        p = ((2 * ll - 1) * x * p1 - (ll + m - 1) * p2) / (ll - m)
        p2, p1 = p1, p
    return p1


def real_sph_harm(l: int, m: int, xyz):
    """Real orthonormal spherical harmonic Y_lm at the directions of xyz [...,3].

    m > 0 uses cos(m*phi), m < 0 uses sin(|m|*phi); normalised so that the
    integral of Y_lm**2 over the unit sphere is 1."""
    xyz = np.asarray(xyz, dtype=np.float64)
    r = np.linalg.norm(xyz, axis=-1)
    ct = xyz[..., 2] / r
    ph = np.arctan2(xyz[..., 1], xyz[..., 0])
    am = abs(m)
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    P = _assoc_legendre(l, am, ct)
    if m == 0:
        return norm * P
    if m > 0:
        return math.sqrt(2.0) * norm * P * np.cos(am * ph)
    return math.sqrt(2.0) * norm * P * np.sin(am * ph)


def bump_sphere(level: int, seed: int, n_modes: int = 8, lmax: int = 4, amp: float = 0.1):
    """Icosphere with radial displacement r = 1 + amp * sum_s a_s Y_{l_s m_s}.

    The n_modes (l, m) pairs are drawn without replacement from the
    (lmax+1)**2 real harmonics with l <= lmax, the a_s are N(0,1); a draw with
    min r < 0.5 is rejected and redrawn from the same generator, so the
    surface stays star-shaped.  Returns (V, T, modes) where modes lists
    (l, m, a)."""
    V, T = icosphere(level)
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = [(l, m) for l in range(lmax + 1) for m in range(-l, l + 1)]
    while True:
        idx = rng.choice(len(pairs), size=n_modes, replace=False)
        a = rng.standard_normal(n_modes)
        r = np.ones(V.shape[0])
        for k, i in enumerate(idx):
            l, m = pairs[i]
            r = r + amp * a[k] * real_sph_harm(l, m, V)
        if r.min() >= 0.5:
            break
    modes = [(pairs[i][0], pairs[i][1], float(a[k])) for k, i in enumerate(idx)]
    return np.ascontiguousarray(V * r[:, None]), T, modes


def stretch(V, scales):
    """Axis-aligned affine stretch x -> diag(scales) x."""
    return np.ascontiguousarray(V * np.asarray(scales, dtype=np.float64)[None, :])


def _unit_dirs(rng, n):
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1)[:, None]


def point_sources(seed: int, n: int, rmin: float = 2.0, rmax: float = 4.0, scales=None, margin: float = 1.1):
    """n exterior point sources with |p| uniform in [rmin, rmax] and uniformly
    distributed direction.  With `scales`, a point inside the stretched
    ellipsoid grown by `margin` (sum (p_a/s_a)^2 <= margin^2) is redrawn."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n:
        d = _unit_dirs(rng, 1)[0]
        p = d * rng.uniform(rmin, rmax)
        if scales is not None and ((p / np.asarray(scales)) ** 2).sum() <= margin ** 2:
            continue
        out.append(p)
    return np.array(out, dtype=np.float64).reshape(n, 3)


def exterior_points(seed: int, n: int, radius: float):
    """n points on the sphere of the given radius (normalised Gaussian directions)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(_unit_dirs(rng, n) * radius)


def interior_points(seed: int, n: int, rmax: float = 0.5):
    """n points uniformly distributed in the ball |x| <= rmax."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = _unit_dirs(rng, n)
    r = rmax * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    return np.ascontiguousarray(d * r[:, None])


def config(name: str):
    """Workload recipes (geometry + sources) with fixed seeds.

    small      : unit icosphere level 4 (5,120 panels), source p = (3,0,0)
    precision  : bumped icosphere level 7 (327,680 panels), 8 harmonics, p = (3,0,0)
    large      : unit icosphere level 8 (1,310,720 panels), 16 sources |p| in [2,4]
    differentiation / differentiation<L> :
                 unit icosphere level 6 (or L), Dirichlet data from p = (3,0,0),
                 1,024 evaluation points on the sphere of radius 2.5
                 (normalised Gaussian directions) and the target field of a
                 point source at (0,0,3) there
    batching / batching<G> :
                 64 (or G) icospheres of levels drawn uniformly from 3..6, each
                 stretched by axis scales log-uniform in [0.5, 2], with 4
                 exterior point sources each (|p| in [2, 4], outside the
                 stretched ellipsoid grown by 1.1); ACA eps = 1e-5
    level<L>   : unit icosphere of level L with p = (3,0,0) (parity ladders)
    """
    if name.startswith("batching"):
        # batching / batching<G>: G geometries (default 64)
        G = int(name[len("batching"):] or 64)
        rng = np.random.Generator(np.random.PCG64(MASTER_SEED + 3))
        levels = rng.integers(3, 7, size=G)
        Vs, Ts, offs, srcs, scales = [], [], [0], [], []
        nv = 0
        for g in range(G):
            V, T = icosphere(int(levels[g]))
            sc = np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=3))
            V = stretch(V, sc)
            Vs.append(V)
            Ts.append(T + nv)
            nv += V.shape[0]
            offs.append(offs[-1] + T.shape[0])
            srcs.append(point_sources(int(rng.integers(1 << 31)), 4, scales=sc))
            scales.append(sc)
        return dict(V=np.ascontiguousarray(np.concatenate(Vs)), T=np.ascontiguousarray(np.concatenate(Ts)),
                    tri_offsets=np.array(offs, dtype=np.int64), sources=np.stack(srcs), levels=levels,
                    scales=np.array(scales), leaf_size=64, eta=1.5, aca_eps=1e-5)
    if name.startswith("differentiation"):
        L = int(name[len("differentiation"):] or 6)
        V, T = icosphere(L)
        pts = exterior_points(MASTER_SEED + 4, 1024, 2.5)
        return dict(V=V, T=T, sources=np.array([[3.0, 0.0, 0.0]]), leaf_size=64, eta=1.5, aca_eps=1e-6,
                    points=pts, target_source=np.array([0.0, 0.0, 3.0]))
    if name == "small":
        V, T = icosphere(4)
        return dict(V=V, T=T, sources=np.array([[3.0, 0.0, 0.0]]), leaf_size=64, eta=1.5, aca_eps=1e-6)
    if name == "precision":
        V, T, modes = bump_sphere(7, MASTER_SEED + 2)
        return dict(V=V, T=T, sources=np.array([[3.0, 0.0, 0.0]]), leaf_size=64, eta=1.5, aca_eps=1e-7, modes=modes)
    if name == "large":
        V, T = icosphere(8)
        return dict(V=V, T=T, sources=point_sources(MASTER_SEED + 5, 16), leaf_size=128, eta=1.5, aca_eps=1e-6)
    if name.startswith("bumped"):
        L = int(name[len("bumped"):])
        V, T, modes = bump_sphere(L, MASTER_SEED + 2)
        return dict(V=V, T=T, sources=np.array([[3.0, 0.0, 0.0]]), leaf_size=64, eta=1.5, aca_eps=1e-7, modes=modes)
    if name.startswith("level"):
        L = int(name[len("level"):])
        V, T = icosphere(L)
        return dict(V=V, T=T, sources=np.array([[3.0, 0.0, 0.0]]), leaf_size=64, eta=1.5, aca_eps=1e-6)
    raise KeyError(name)
