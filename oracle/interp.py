"""Directional Chebyshev interpolation: the analytic DH^2 matrix (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

Follows Section 2 of the paper:

* tensor interpolation points xi_{t,nu} in the box B_t and tensor Lagrange
  polynomials L_{t,nu}; "order m" means m points per axis, k = m^3
  (Section 5: "order m = 4 ... k = 4^3 = 64").  First-kind Chebyshev nodes
  mid + half cos(pi (2j+1) / (2m)), tensor index nu = nu_x + m nu_y + m^2 nu_z.
  Degenerate axes (zero box thickness) get their half-width padded to at least
  1e-3 times the largest half-width of the box (paper silent).
* modified Lagrange L_{tc,nu}(x) = exp(i kappa <x,c>) L_{t,nu}(x);
  leaf bases v_{tc,i nu} = int phi_i L_{tc,nu} by the 3-point rule;
  couplings s_{b,nu mu} = g_c(xi_{t,nu}, xi_{s,mu})          (Eq. matrix_apx)
* transfer matrices e_{t'c, nu' nu} = exp(i kappa <xi_{t' nu'}, c - c'>) L_{t,nu}(xi_{t' nu'})
  with c' = sd(c)                                             (Eq. nested_apx)
  so that V_tc restricted to t' is V_{t'c'} E_{t'c}          (Eq. nested)
* the column basis uses the same modified Lagrange form, so W = V.

Pins (tests/test_oracle_interp.py): Lagrange polynomials are the Kronecker
delta on the nodes and reproduce x^a y^b z^c, a,b,c <= m-1, to rounding; with
c = c' = 0 the nested property holds to rounding (polynomial reproduction);
with c != 0 the nested error decays as m grows (convergence, not a pin); the
expanded interpolated DH^2 equals the blockwise sum V S V^* + nearfield by
brute force.  The distance of this approximation from the dense matrix G is
interpolation error: parity unpinned as a value (it is measured and reported).
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import Discretisation, helmholtz_c
from .structure import BlockTree, ClusterTree, Directions, PairIndex


class ChebyshevBoxes:
    """Per-cluster 1-D Chebyshev nodes (nc, 3, m) on the padded bounding boxes."""

    def __init__(self, tree: ClusterTree, m: int):
        self.m = m
        mid = (tree.lo + tree.hi) * 0.5
        half = (tree.hi - tree.lo) * 0.5
        hmax = half.max(axis=1, keepdims=True)
        half = np.maximum(half, 1e-3 * hmax)
        j = np.arange(m)
        ref = np.cos(math.pi * (2 * j + 1) / (2 * m))            # (m,)
        self.nodes = mid[:, :, None] + half[:, :, None] * ref[None, None, :]

    def lagrange_1d(self, t, axis, x):
        """l_{t,axis,j}(x) for all j: array (len(x), m), product form."""
        xi = self.nodes[t, axis]
        x = np.asarray(x, dtype=np.float64)
        out = np.ones((len(x), self.m))
        for j in range(self.m):
            for i in range(self.m):
                if i != j:
                    out[:, j] *= (x - xi[i]) / (xi[j] - xi[i])
        return out

    def lagrange(self, t, x):
        """Tensor L_{t,nu}(x) for points x (p, 3): array (p, k), nu = nx + m ny + m^2 nz."""
        lx = self.lagrange_1d(t, 0, x[:, 0])
        ly = self.lagrange_1d(t, 1, x[:, 1])
        lz = self.lagrange_1d(t, 2, x[:, 2])
        return (lz[:, :, None, None] * ly[:, None, :, None] * lx[:, None, None, :]).reshape(len(x), -1)

    def points(self, t):
        """Tensor interpolation points xi_{t,nu}, shape (k, 3)."""
        m = self.m
        nz, ny, nx = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
        return np.stack([self.nodes[t, 0][nx.ravel()], self.nodes[t, 1][ny.ravel()],
                         self.nodes[t, 2][nz.ravel()]], axis=1)


class InterpolatedDH2:
    """The analytic DH^2 matrix of Section 2 with all matrices stored (O2)."""

    def __init__(self, disc: Discretisation, tree: ClusterTree, dirs: Directions,
                 blocks: BlockTree, kappa: float, m: int):
        self.disc, self.tree, self.dirs, self.blocks = disc, tree, dirs, blocks
        self.kappa, self.m, self.k = kappa, m, m ** 3
        self.cheb = ChebyshevBoxes(tree, m)
        self.pairs = PairIndex(tree, dirs, blocks)

    def direction(self, t, c):
        return self.dirs.dirs[self.tree.level[t]][c]

    def leaf_basis(self, t, c):
        """V_tc for a leaf t: (#t, k), rows in cluster order (3-point rule)."""
        idx = self.tree.indices(t)
        x = self.disc.x3[idx]                                   # (#t, 3, 3)
        w = self.disc.w3[idx]                                   # (#t, 3)
        cvec = self.direction(t, c)
        pts = x.reshape(-1, 3)
        lag = self.cheb.lagrange(t, pts).reshape(len(idx), 3, -1)
        wave = np.exp(1j * self.kappa * (pts @ cvec)).reshape(len(idx), 3)
        return np.einsum("iq,iq,iqn->in", w, wave, lag)

    def transfer(self, tson, c):
        """E_{t'c}: (k, k) for the son t' of t and c in D_t; c' = sd(c) (Eq. nested_apx)."""
        t = self.tree.parent[tson]
        l = self.tree.level[t]
        cvec = self.dirs.dirs[l][c]
        cson = self.dirs.dirs[l + 1][self.dirs.sd[l][c]]
        xi = self.cheb.points(tson)                             # (k, 3)
        wave = np.exp(1j * self.kappa * (xi @ (cvec - cson)))   # (k,)
        return wave[:, None] * self.cheb.lagrange(t, xi)

    def coupling(self, b):
        """S_b = g_c(xi_t, xi_s): (k, k) for admissible block b = (t, s, c)."""
        t, s, c = self.blocks.adm[b]
        cvec = self.direction(t, c)
        xt = self.cheb.points(t)
        xs = self.cheb.points(s)
        return helmholtz_c(xt[:, None, :], xs[None, :, :], self.kappa, cvec)

    def son_direction(self, t, c):
        return int(self.dirs.sd[self.tree.level[t]][c])

    def full_basis(self, t, c):
        """Expanded V_tc (#t, k) through Eq. (nested): used by tests on tiny meshes."""
        tr = self.tree
        if tr.is_leaf(t):
            return self.leaf_basis(t, c)
        c1 = self.son_direction(t, c)
        return np.vstack([self.full_basis(ts, c1) @ self.transfer(ts, c)
                          for ts in (tr.son0[t], tr.son1[t])])

    def nearfield_block(self, t, s):
        """G restricted to t x s (cluster order), the same quadrature as the dense G."""
        return self.disc.entries(self.tree.indices(t), self.tree.indices(s), self.kappa)

    def to_dense(self):
        """Expanded interpolated matrix in ORIGINAL numbering (tiny meshes only)."""
        n = self.tree.n
        A = np.zeros((n, n), dtype=np.complex128)
        for (t, s) in self.blocks.near:
            A[np.ix_(self.tree.indices(t), self.tree.indices(s))] = self.nearfield_block(t, s)
        for b, (t, s, c) in enumerate(self.blocks.adm):
            Vt = self.full_basis(t, c)
            Vs = self.full_basis(s, c)
            A[np.ix_(self.tree.indices(t), self.tree.indices(s))] = Vt @ self.coupling(b) @ Vs.conj().T
        return A

    def matvec(self, x):
        """y = G_DH2 x block by block (x, y in original numbering)."""
        tr = self.tree
        y = np.zeros(tr.n, dtype=np.complex128)
        for (t, s) in self.blocks.near:
            y[tr.indices(t)] += self.nearfield_block(t, s) @ x[tr.indices(s)]
        for b, (t, s, c) in enumerate(self.blocks.adm):
            Vt = self.full_basis(t, c)
            Vs = self.full_basis(s, c)
            y[tr.indices(t)] += Vt @ (self.coupling(b) @ (Vs.conj().T @ x[tr.indices(s)]))
        return y
