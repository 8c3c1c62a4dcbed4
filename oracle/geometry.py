"""Kernel, quadrature and dense Galerkin matrix (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

* Helmholtz kernel g(x,y) = exp(i kappa |x-y|) / (4 pi |x-y|)   (Eq. 1)
* directional remainder g_c(x,y) = exp(i kappa (|x-y| - <x-y,c>)) / (4 pi |x-y|)
                                                                (Section 2, plane-wave split)
* Galerkin entries g_ij = int phi_i int g phi_j               (Eq. 2) with
  piecewise-constant phi_i = indicator of triangle i (Section 5).

Quadrature (the paper uses Sauter-Erichsen-Schwab rules, Section 5; this
oracle reads the simpler rule fixed for the workloads): the 3-point interior
rule, barycentric (2/3,1/6,1/6) and permutations with weights |T|/3, exact for
degree 2; for i == j the x-integral uses the 7-point degree-5 rule of Radon
(Stroud T2:5-1) against the 3-point rule in y, so the node sets are disjoint
and the singular integrand stays finite.

Pins (tests/test_oracle_geometry.py): rule exactness on monomials against the
closed form int_T x^a y^b = a! b! / (a+b+2)! on the reference triangle; weight
sums = |T|; kernel closed forms (kappa = 0 is the Laplace kernel, g_0 = g);
symmetry g_ij = g_ji off the diagonal; kappa = 0 gives a real matrix.
"""
from __future__ import annotations

import math

import numpy as np

FOUR_PI = 4.0 * math.pi

# 3-point interior rule: barycentric coordinates, weights relative to |T|.
BARY3 = np.array(
    [[2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0],
     [1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0],
     [1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0]]
)
W3 = np.array([1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0])

# 7-point degree-5 rule (Radon 1948; Stroud T2:5-1), weights relative to |T|.
_s15 = math.sqrt(15.0)
_a1, _b1 = (6.0 - _s15) / 21.0, (9.0 + 2.0 * _s15) / 21.0
_a2, _b2 = (6.0 + _s15) / 21.0, (9.0 - 2.0 * _s15) / 21.0
BARY7 = np.array(
    [[1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0],
     [_b1, _a1, _a1], [_a1, _b1, _a1], [_a1, _a1, _b1],
     [_b2, _a2, _a2], [_a2, _b2, _a2], [_a2, _a2, _b2]]
)
W7 = np.array(
    [9.0 / 40.0]
    + [(155.0 - _s15) / 1200.0] * 3
    + [(155.0 + _s15) / 1200.0] * 3
)


def helmholtz(x, y, kappa):
    """g(x,y) of Eq. 1 for arrays of points (..., 3)."""
    d = x - y
    r = np.sqrt(np.sum(d * d, axis=-1))
    return np.exp(1j * kappa * r) / (FOUR_PI * r)


def helmholtz_c(x, y, kappa, c):
    """Remainder g_c after splitting off exp(i kappa <x-y, c>) (Section 2)."""
    d = x - y
    r = np.sqrt(np.sum(d * d, axis=-1))
    dc = np.sum(d * np.asarray(c), axis=-1)
    return np.exp(1j * kappa * (r - dc)) / (FOUR_PI * r)


def triangle_areas(vertices, triangles):
    v0, v1, v2 = (vertices[triangles[:, j]] for j in range(3))
    cr = np.cross(v1 - v0, v2 - v0)
    return 0.5 * np.sqrt(np.sum(cr * cr, axis=1))


def quad_points(vertices, triangles, bary):
    """Quadrature nodes x = l0 v0 + l1 v1 + l2 v2, shape (n, q, 3)."""
    v0, v1, v2 = (vertices[triangles[:, j]] for j in range(3))
    return (bary[None, :, 0, None] * v0[:, None, :]
            + bary[None, :, 1, None] * v1[:, None, :]
            + bary[None, :, 2, None] * v2[:, None, :])


class Discretisation:
    """Piecewise-constant Galerkin discretisation of the single layer operator."""

    def __init__(self, vertices, triangles):
        self.vertices = np.asarray(vertices, dtype=np.float64)
        self.triangles = np.asarray(triangles, dtype=np.int64)
        self.n = len(self.triangles)
        self.area = triangle_areas(self.vertices, self.triangles)
        self.x3 = quad_points(self.vertices, self.triangles, BARY3)   # (n,3,3)
        self.w3 = self.area[:, None] * W3[None, :]                    # (n,3)
        self.x7 = quad_points(self.vertices, self.triangles, BARY7)   # (n,7,3)
        self.w7 = self.area[:, None] * W7[None, :]                    # (n,7)

    def entries(self, rows, cols, kappa):
        """g_ij (Eq. 2) for the index grid rows x cols (original numbering)."""
        rows = np.asarray(rows)
        cols = np.asarray(cols)
        xi = self.x3[rows][:, None, :, None, :]      # (R,1,3,1,3)
        yj = self.x3[cols][None, :, None, :, :]      # (1,C,1,3,3)
        w = self.w3[rows][:, None, :, None] * self.w3[cols][None, :, None, :]
        diag = rows[:, None] == cols[None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            # the 3x3 rule is singular on the diagonal; those entries are replaced below
            out = np.sum(w * helmholtz(xi, yj, kappa), axis=(2, 3))
        if diag.any():
            ri, ci = np.nonzero(diag)
            i = rows[ri]
            x = self.x7[i][:, :, None, :]            # (D,7,1,3)
            y = self.x3[i][:, None, :, :]            # (D,1,3,3)
            wd = self.w7[i][:, :, None] * self.w3[i][:, None, :]
            out[ri, ci] = np.sum(wd * helmholtz(x, y, kappa), axis=(1, 2))
        return out

    def dense(self, kappa, chunk=None):
        """The full Galerkin matrix G (n x n), ground truth for the matvec error."""
        n = self.n
        chunk = chunk or max(1, (1 << 21) // n)
        G = np.empty((n, n), dtype=np.complex128)
        cols = np.arange(n)
        for r0 in range(0, n, chunk):
            rows = np.arange(r0, min(n, r0 + chunk))
            G[rows] = self.entries(rows, cols, kappa)
        return G

    def dense_rows_matvec(self, rows, x, kappa, chunk=None):
        """(G x)[rows] assembled row by row (sampled dense rows for big meshes)."""
        rows = np.asarray(rows)
        chunk = chunk or max(1, (1 << 21) // self.n)
        out = np.empty(len(rows), dtype=np.complex128)
        cols = np.arange(self.n)
        for r0 in range(0, len(rows), chunk):
            rr = rows[r0:r0 + chunk]
            out[r0:r0 + chunk] = self.entries(rr, cols, kappa) @ x
        return out
