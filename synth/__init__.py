"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only *generates inputs*: surface meshes shaped like the paper's
test geometries (Section 5: unit sphere and unit cube, regularly refined flat
triangles) and seeded complex right-hand sides.  It contains none of the
method's arithmetic (no kernel, quadrature, clustering or compression).

Mesh conventions (fixed so that every consumer sees the same input):

* ``icosphere(L)``: the 12 vertices of the regular icosahedron, normalised,
  then ``L`` rounds of regular 1:4 refinement.  New midpoint vertices are
  created in face order, each edge once (key = sorted vertex pair) and
  projected onto the unit sphere by ``v / ||v||``.  Each face (a, b, c) is
  replaced by (a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca).
  ``20 * 4**L`` triangles: L=3 -> 1280, L=5 -> 20480, L=6 -> 81920.
* ``ellipsoid(L, axes)``: the icosphere scaled per axis, x -> (a x, b y, c z).
* ``cube(q)``: surface of [-1/2, 1/2]^3, q x q squares per face, each square
  split along a fixed diagonal: ``12 q**2`` triangles.
* ``random_vector(n, seed)``: N(0,1) + i N(0,1) from numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

__all__ = ["icosphere", "ellipsoid", "cube", "random_vector", "batch_meshes", "point_cloud"]


def _icosahedron():
    p = (1.0 + np.sqrt(5.0)) / 2.0
    v = np.array(
        [
            [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
            [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
            [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
        ],
        dtype=np.float64,
    )
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int32,
    )
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosphere(level: int):
    """Unit-sphere triangulation with ``20 * 4**level`` flat triangles."""
    verts, faces = _icosahedron()
    verts = [tuple(x) for x in verts]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}
        new_faces = []

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                m = (np.asarray(verts[a]) + np.asarray(verts[b])) * 0.5
                m = m / np.sqrt(m @ m)
                idx = len(verts)
                verts.append(tuple(m))
                cache[key] = idx
            return idx

        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = np.asarray(new_faces, dtype=np.int32)
    return np.asarray(verts, dtype=np.float64), np.ascontiguousarray(faces, dtype=np.int32)


def ellipsoid(level: int, axes):
    v, f = icosphere(level)
    return v * np.asarray(axes, dtype=np.float64)[None, :], f


def cube(q: int):
    """Surface of [-1/2, 1/2]^3 with ``12 q**2`` triangles."""
    verts: list[tuple[float, float, float]] = []
    faces: list[tuple[int, int, int]] = []
    g = np.linspace(-0.5, 0.5, q + 1)
    for axis in range(3):
        for sign in (1.0, -1.0):
            b, c = [a for a in range(3) if a != axis]
            base = len(verts)
            for i in range(q + 1):
                for j in range(q + 1):
                    p = [0.0, 0.0, 0.0]
                    p[axis] = 0.5 * sign
                    p[b] = g[i]
                    p[c] = g[j]
                    verts.append(tuple(p))
            for i in range(q):
                for j in range(q):
                    v00 = base + i * (q + 1) + j
                    v01 = v00 + 1
                    v10 = v00 + (q + 1)
                    v11 = v10 + 1
                    faces.append((v00, v10, v11))
                    faces.append((v00, v11, v01))
    return np.asarray(verts, dtype=np.float64), np.asarray(faces, dtype=np.int32)


def point_cloud(n: int, seed: int):
    """Seeded points on the unit sphere (used by point-mode tests)."""
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((n, 3))
    return p / np.linalg.norm(p, axis=1, keepdims=True)


def random_vector(n: int, seed: int, count: int | None = None):
    """Seeded complex vector(s) N(0,1) + i N(0,1), complex128."""
    rng = np.random.default_rng(seed)
    shape = (n,) if count is None else (count, n)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def batch_meshes(count: int, seed: int):
    """The batched workload: spheres and ellipsoids of 1280-20480 triangles.

    Per mesh: refinement level L uniform in {3,4,5}; ellipsoid with
    probability 1/2 with semi-axes U[0.5, 2]^3; wave number U[4, 16].
    Returns a list of ``(vertices, triangles, kappa)``.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        level = int(rng.integers(3, 6))
        is_ell = bool(rng.random() < 0.5)
        axes = rng.uniform(0.5, 2.0, size=3) if is_ell else np.ones(3)
        kappa = float(rng.uniform(4.0, 16.0))
        v, f = ellipsoid(level, axes)
        out.append((v, f, kappa))
    return out


def directional_meshes(count: int, seed: int):
    """Meshes whose admissible blocks reach directional levels at eta1 = 10: spheres and
    ellipsoids of 20480 triangles (refinement level 5; ellipsoid with probability 1/2,
    semi-axes U[0.8, 1.25]^3) with wave number U[28, 40].  Returns (vertices, triangles, kappa)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        is_ell = bool(rng.random() < 0.5)
        axes = rng.uniform(0.8, 1.25, size=3) if is_ell else np.ones(3)
        kappa = float(rng.uniform(28.0, 40.0))
        v, f = ellipsoid(5, axes)
        out.append((v, f, kappa))
    return out
