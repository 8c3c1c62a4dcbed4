"""Double-layer potential of the Helmholtz equation: kernel and dense Galerkin matrix (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).  The paper's second operator (Section
5, its table for the double-layer potential): the same Galerkin discretisation as the single
layer operator with the kernel differentiated along the normal of the y element,

    d/dn_y g(x, y) = exp(i kappa r) (1 - i kappa r) <x - y, n_y> / (4 pi r^3),  r = |x - y|,

(from g(x, y) = exp(i kappa r) / (4 pi r), dr/dn_y = -<x - y, n_y> / r).

* normals: n_j = (v1 - v0) x (v2 - v0) / |.|, the right-hand rule of the vertex order
  (outward for the icospheres and ellipsoids of ``synth``);
* entries k_ij = int phi_i(x) int d/dn_y g(x, y) phi_j(y) by the 3 x 3 interior rule of
  ``oracle.geometry``; on the diagonal x - y lies in the plane of the flat triangle, so the
  integrand and k_ii vanish;
* ``potential(points)`` = int_Gamma d/dn_y g(x, y) dy (density 1) by the 3-point rule.

Pins (tests/test_oracle_double_layer.py): the kernel equals central finite differences of
g along n_y; for kappa = 0 the potential of the constant density is -1 inside the closed
surface and 0 outside (Gauss's solid-angle identity, exact for the closed polyhedron, so only
quadrature error remains and it falls under refinement); k_ii = 0; kappa = 0 gives a real
matrix.
"""
from __future__ import annotations

import numpy as np

from .geometry import FOUR_PI, Discretisation


def triangle_normals(vertices, triangles):
    v = np.asarray(vertices, dtype=np.float64)
    t = np.asarray(triangles)
    n = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def dlp_kernel(x, y, ny, kappa):
    """d/dn_y g(x, y) for arrays of points (..., 3) and normals (..., 3)."""
    d = x - y
    r = np.sqrt(np.sum(d * d, axis=-1))
    dn = np.sum(d * ny, axis=-1)
    return np.exp(1j * kappa * r) * (1.0 - 1j * kappa * r) * dn / (FOUR_PI * r ** 3)


class DoubleLayer:
    """Piecewise-constant Galerkin matrix of the double-layer potential."""

    def __init__(self, vertices, triangles):
        self.disc = Discretisation(vertices, triangles)
        self.normals = triangle_normals(vertices, triangles)
        self.n = self.disc.n

    def entries(self, rows, cols, kappa):
        """k_ij for the index grid rows x cols (original numbering); 0 on the diagonal."""
        rows, cols = np.asarray(rows), np.asarray(cols)
        d = self.disc
        xi = d.x3[rows][:, None, :, None, :]           # (R,1,3,1,3)
        yj = d.x3[cols][None, :, None, :, :]           # (1,C,1,3,3)
        nj = self.normals[cols][None, :, None, None, :]
        w = d.w3[rows][:, None, :, None] * d.w3[cols][None, :, None, :]
        diag = rows[:, None] == cols[None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            out = np.sum(w * dlp_kernel(xi, yj, nj, kappa), axis=(2, 3))
        out[diag] = 0.0
        return out

    def dense(self, kappa):
        idx = np.arange(self.n)
        return self.entries(idx, idx, kappa)

    def potential(self, points, kappa):
        """int_Gamma d/dn_y g(x, y) dy at each point (density 1), 3-point rule per element."""
        d = self.disc
        x = np.asarray(points, dtype=np.float64)[:, None, None, :]     # (P,1,1,3)
        y = d.x3[None, :, :, :]                                          # (1,n,3,3)
        ny = self.normals[None, :, None, :]
        return np.sum(d.w3[None, :, :] * dlp_kernel(x, y, ny, kappa), axis=(1, 2))
