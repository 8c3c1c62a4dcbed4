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

* ``InterpolatedDLP``: its directional interpolation (rows V_tc as for the single layer,
  columns W_sc from the normal derivative of the modified Lagrange polynomials, the same
  transfers and couplings), stored and expanded like ``oracle.interp.InterpolatedDH2``.
* ``RecompressionDLP``: Section 3.2 with separate row and column basis weights.

Pins (tests/test_oracle_double_layer.py): the kernel equals central finite differences of
g along n_y; for kappa = 0 the potential of the constant density is -1 inside the closed
surface and 0 outside (Gauss's solid-angle identity, exact for the closed polyhedron, so only
quadrature error remains and it falls under refinement); Green's representation formula of a
plane wave inside the sphere; k_ii = 0; kappa = 0 gives a real matrix.  Interpolated form:
gradients of the tensor Lagrange polynomials reproduce gradients of polynomials of degree
<= m - 1 per axis; W applied to nodal values of a cubic equals the integral of its normal
derivative (closed form by the 7-point rule); the blockwise product equals the expanded
matrix by brute force; the distance to the dense matrix falls as m grows (convergence, not
a pin).  Recompression: R^* R = V^* V and R_W^* R_W = W^* W through Eq. (nested); new bases
orthonormal; every block within eps sqrt(2 (p + 1)) of the interpolated one (the Pythagoras
chain of Section 3.1); the product equals the expanded recompressed matrix.
"""
from __future__ import annotations

import numpy as np

from .geometry import FOUR_PI, Discretisation
from .interp import InterpolatedDH2
from .recompress import RANK_BLOCKREL, Recompression, qr_r


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


# --------------------------------------------------------------------------- interpolated DLP


def lagrange_1d_derivative(nodes, x):
    """l_j'(x) for the 1-D Lagrange basis on `nodes`: (len(x), m), product form
    l_j'(x) = sum_{k != j} 1 / (xi_j - xi_k) prod_{i != j, k} (x - xi_i) / (xi_j - xi_i)."""
    m = len(nodes)
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((len(x), m))
    for j in range(m):
        for k in range(m):
            if k == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[k]))
            for i in range(m):
                if i != j and i != k:
                    term *= (x - nodes[i]) / (nodes[j] - nodes[i])
            out[:, j] += term
    return out


class InterpolatedDLP(InterpolatedDH2):
    """The analytic DH^2 matrix of the double-layer potential: rows as for the single layer
    (V_tc), columns with the normal derivative of the modified Lagrange polynomials,
        w_{sc, j mu} = int phi_j d/dn_j [exp(i kappa <y, c>) L_{s,mu}(y)] dy
                     = int phi_j exp(i kappa <y, c>) (i kappa <n_j, c> L_{s,mu}(y) + <n_j, grad L_{s,mu}(y)>) dy,
    so that a block is V_tc S_b W_sc^* (the y factor of the expansion of g is
    exp(-i kappa <y, c>) L_{s,mu}(y), differentiated along n_y).  The transfers are those
    of V: the normal derivative is linear and acts after the nested expansion."""

    def __init__(self, layer: DoubleLayer, tree, dirs, blocks, kappa, m):
        super().__init__(layer.disc, tree, dirs, blocks, kappa, m)
        self.layer = layer

    def lagrange_grad(self, t, x):
        """grad L_{t,nu}(x) for points x (p, 3): array (p, k, 3), nu = nx + m ny + m^2 nz."""
        c = self.cheb
        l = [c.lagrange_1d(t, a, x[:, a]) for a in range(3)]
        d = [lagrange_1d_derivative(c.nodes[t, a], x[:, a]) for a in range(3)]

        def tensor(fx, fy, fz):
            return (fz[:, :, None, None] * fy[:, None, :, None] * fx[:, None, None, :]).reshape(len(x), -1)

        return np.stack([tensor(d[0], l[1], l[2]), tensor(l[0], d[1], l[2]), tensor(l[0], l[1], d[2])], axis=2)

    def leaf_col_basis(self, s, c):
        """W_sc for a leaf s: (#s, k), rows in cluster order (3-point rule)."""
        idx = self.tree.indices(s)
        x = self.disc.x3[idx]
        w = self.disc.w3[idx]
        nrm = self.layer.normals[idx]                                  # (#s, 3)
        cvec = self.direction(s, c)
        pts = x.reshape(-1, 3)
        npt = np.repeat(nrm, 3, axis=0)                                # normal of each point's element
        lag = self.cheb.lagrange(s, pts)                               # (3#s, k)
        grad = self.lagrange_grad(s, pts)                              # (3#s, k, 3)
        dn = np.einsum("pka,pa->pk", grad, npt) + 1j * self.kappa * (npt @ cvec)[:, None] * lag
        wave = np.exp(1j * self.kappa * (pts @ cvec))
        vals = (wave[:, None] * dn).reshape(len(idx), 3, -1)
        return np.einsum("iq,iqn->in", w, vals)

    def full_col_basis(self, s, c):
        tr = self.tree
        if tr.is_leaf(s):
            return self.leaf_col_basis(s, c)
        c1 = self.son_direction(s, c)
        return np.vstack([self.full_col_basis(ss, c1) @ self.transfer(ss, c)
                          for ss in (tr.son0[s], tr.son1[s])])

    def nearfield_block(self, t, s):
        return self.layer.entries(self.tree.indices(t), self.tree.indices(s), self.kappa)

    def to_dense(self):
        n = self.tree.n
        A = np.zeros((n, n), dtype=np.complex128)
        for (t, s) in self.blocks.near:
            A[np.ix_(self.tree.indices(t), self.tree.indices(s))] = self.nearfield_block(t, s)
        for b, (t, s, c) in enumerate(self.blocks.adm):
            A[np.ix_(self.tree.indices(t), self.tree.indices(s))] = (
                self.full_basis(t, c) @ self.coupling(b) @ self.full_col_basis(s, c).conj().T)
        return A

    def matvec(self, x):
        tr = self.tree
        y = np.zeros(tr.n, dtype=np.complex128)
        for (t, s) in self.blocks.near:
            y[tr.indices(t)] += self.nearfield_block(t, s) @ x[tr.indices(s)]
        for b, (t, s, c) in enumerate(self.blocks.adm):
            Vt = self.full_basis(t, c)
            Ws = self.full_col_basis(s, c)
            y[tr.indices(t)] += Vt @ (self.coupling(b) @ (Ws.conj().T @ x[tr.indices(s)]))
        return y


# --------------------------------------------------------------------------- recompression

class RecompressionDLP(Recompression):
    """Section 3.2 for a DH^2 matrix whose column basis differs from its row basis
    (W != V, the double-layer potential): the same steps with basis weights R from V and
    R_W from W (Eq. basis_weights_def for each basis), block norms |R_tc S_b R_W,sc^*|_F,
    row total weights stacking R_W,sc S_b^* and column total weights stacking R_tc S_b,
    and the row truncation on V, the column truncation on W."""

    def __init__(self, dh2: InterpolatedDLP, eps: float, rule=RANK_BLOCKREL):
        self.dh2, self.eps, self.rule = dh2, eps, rule
        self.tree, self.pairs, self.k = dh2.tree, dh2.pairs, dh2.k
        self._S = {}
        self._E = {}
        self.R = self.weights(dh2.leaf_basis)
        self.RW = self.weights(dh2.leaf_col_basis)
        self.block_norms()
        self.ZR = self.total_weights(rows=True)
        self.ZC = self.total_weights(rows=False)
        self.row = self.truncate_basis(self.ZR, dh2.leaf_basis)
        self.col = self.truncate_basis(self.ZC, dh2.leaf_col_basis)
        self.project()

    def weights(self, leaf):
        tr, P, d = self.tree, self.pairs, self.dh2
        R = {}
        for l in range(tr.depth, -1, -1):
            for t, c in self.active_pairs(l):
                if tr.is_leaf(t):
                    a = leaf(t, c)
                else:
                    c1 = d.son_direction(t, c)
                    a = np.vstack([R[P.tc(ts, c1)] @ self.E(ts, c) for ts in (tr.son0[t], tr.son1[t])])
                R[P.tc(t, c)] = qr_r(a, self.k)
        return R

    def block_norms(self):
        P = self.pairs
        adm = self.dh2.blocks.adm
        self.bnorm = np.zeros(len(adm))
        for b, (t, s, c) in enumerate(adm):
            self.bnorm[b] = np.linalg.norm(self.R[P.tc(t, c)] @ self.S(b) @ self.RW[P.tc(s, c)].conj().T)

    def total_weights(self, rows: bool):
        tr, P = self.tree, self.pairs
        adm = self.dh2.blocks.adm
        Z = {}
        for l in range(tr.depth + 1):
            for t, c in self.active_pairs(l):
                tc = P.tc(t, c)
                parts = []
                for b in (P.row[tc] if rows else P.col[tc]):
                    tb, sb, _ = adm[b]
                    if rows:
                        parts.append(self.RW[P.tc(sb, c)] @ self.S(b).conj().T / self.bnorm[b])
                    else:
                        parts.append(self.R[P.tc(tb, c)] @ self.S(b) / self.bnorm[b])
                tp = tr.parent[t]
                if tp >= 0:
                    for cp in P.sd_inverse(tp, c):
                        zp = Z.get(P.tc(tp, cp))
                        if zp is not None and zp.shape[0] > 0:
                            parts.append(zp @ self.E(t, cp).conj().T)
                stack = np.vstack(parts) if parts else np.zeros((0, self.k), dtype=np.complex128)
                Z[tc] = qr_r(stack, self.k)
        return Z

    def truncate_basis(self, Z, leaf):
        """The truncation of Recompression.truncate with the leaf basis `leaf` (V or W)."""
        saved = self.dh2.leaf_basis
        try:
            self.dh2.leaf_basis = leaf
            return Recompression.truncate(self, Z)
        finally:
            self.dh2.leaf_basis = saved
