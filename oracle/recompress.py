"""Algebraic recompression of the interpolated DH^2 matrix (oracle, FP64, Section 3.2).

Test infrastructure only (see ``oracle/__init__``).

Steps, in the paper's order (all pairs (t,c) of the active set, W = V):

1. basis weights R_tc (Eq. basis_weights_def), bottom-up:
   leaf:     V_tc = P R_tc                       (QR)
   non-leaf: [R_{t1c1} E_{t1c}; R_{t2c2} E_{t2c}] = P R_tc   (QR), c_i = sd(c)
   R_tc has min(rows, k) rows (leaves have fewer than k rows).
2. block weights: each admissible block enters with weight 1/||G_b||_F, where
   ||G_b||_F = ||R_tc S_b R_sc^*||_F exactly (reading of the paper's
   "block-wise relative Frobenius norm", Section 5).
3. total weights Z-hat_tc (Eq. recomp_weight_full), top-down:
   Z_tc^* = [ R_sc S_b^* / ||G_b|| for b in row(t,c) ;
              Z-hat_{t+c+} E_{tc+}^*  for c+ in sd^{-1}(c) ]     (stacked rows)
   Z-hat_tc = R-factor of the QR of Z_tc^*.  The column basis repeats this on
   G^* with R_tc S_b / ||G_b|| for b in col(s,c).
4. truncation, bottom-up: leaf A = V_tc Z-hat^*, non-leaf
   A = V-hat Z-hat^* with V-hat = [C_{t1c1} E_{t1c}; C_{t2c2} E_{t2c}]; SVD of A;
   rank k_tc = smallest k with sum_{i>k} sigma_i^2 <= eps^2 (blockwise
   relative: every block carries norm 1), or <= eps^2 sum sigma^2 ("global"
   reading), or, for error control in the spectral norm (Section 5, Table
   "spectral norm"; the best rank-k error in the spectral norm is sigma_{k+1}),
   the smallest k with sigma_{k+1} <= eps on the same weighted matrix; Q = first k_tc left singular vectors (leaf) or
   Q-hat = [F_{t1c}; F_{t2c}] (non-leaf); C_tc = Q^* V (or Q-hat^* V-hat)
   (Eq. C_tc).
5. projection S~_b = C_tc S_b C^W_sc^*  (Lemma "Projections").
6. the recompressed DH^2 matvec: forward transform with the column basis,
   couplings, backward transform with the row basis, plus the nearfield
   (derived from Eq. nested and Eq. vsw; the paper states no matvec).

Pins (tests/test_oracle_recompress.py): R^* R = V^* V with V expanded through
Eq. (nested); V Z-hat^* Z-hat V^* = G_tc G_tc^* for the weighted, explicitly
assembled G_tc (Eq. recomp_weight_full); the singular values of the
Section 3.1 algorithm applied to the explicit G_tc / G-hat_tc equal those of
this Section 3.2 path (the paper's claim that P_tc does not change them);
Q^* Q = I; per-block error of the recompressed against the interpolated
matrix <= eps sqrt(2 (p+1)) ||G_b||; the matvec equals the expanded dense
recompressed matrix.
"""
from __future__ import annotations

import numpy as np

from .interp import InterpolatedDH2

RANK_BLOCKREL = 0
RANK_GLOBAL = 1
RANK_SPECTRAL = 2


def qr_r(a, k):
    """R-factor of a QR factorisation, min(rows, k) x k (numpy / LAPACK)."""
    if a.shape[0] == 0:
        return np.zeros((0, k), dtype=np.complex128)
    return np.linalg.qr(a, mode="r")


def choose_rank(sigma, eps, rule=RANK_BLOCKREL):
    """Smallest k with sum_{i>k} sigma_i^2 <= bound (Section 3.1, Frobenius), or with
    sigma_{k+1} <= eps (spectral norm; sigma sorted descending)."""
    if rule == RANK_SPECTRAL:
        return int(np.count_nonzero(np.asarray(sigma, dtype=np.float64) > eps))
    s2 = sigma.astype(np.float64) ** 2
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])   # tail[k] = sum_{i>=k}
    bound = eps * eps if rule == RANK_BLOCKREL else eps * eps * float(s2.sum())
    for kk in range(len(sigma) + 1):
        if tail[kk] <= bound:
            return kk
    return len(sigma)


class Recompression:
    def __init__(self, dh2: InterpolatedDH2, eps: float, rule=RANK_BLOCKREL):
        self.dh2, self.eps, self.rule = dh2, eps, rule
        self.tree, self.pairs, self.k = dh2.tree, dh2.pairs, dh2.k
        self._S = {}
        self._E = {}
        self.basis_weights()
        self.block_norms()
        self.ZR = self.total_weights(rows=True)
        self.ZC = self.total_weights(rows=False)
        self.row = self.truncate(self.ZR)
        self.col = self.truncate(self.ZC)
        self.project()

    # -- cached analytic pieces ------------------------------------------------
    def S(self, b):
        if b not in self._S:
            self._S[b] = self.dh2.coupling(b)
        return self._S[b]

    def E(self, tson, c):
        key = (int(tson), int(c))
        if key not in self._E:
            self._E[key] = self.dh2.transfer(tson, c)
        return self._E[key]

    def active_pairs(self, level):
        tr, P = self.tree, self.pairs
        for t in range(tr.level_start[level], tr.level_start[level + 1]):
            for c in range(P.count[t]):
                if P.active[P.base[t] + c]:
                    yield int(t), int(c)

    # -- step 1 ----------------------------------------------------------------
    def basis_weights(self):
        tr, P, d = self.tree, self.pairs, self.dh2
        self.R = {}
        for l in range(tr.depth, -1, -1):
            for t, c in self.active_pairs(l):
                if tr.is_leaf(t):
                    a = d.leaf_basis(t, c)
                else:
                    c1 = d.son_direction(t, c)
                    a = np.vstack([self.R[P.tc(ts, c1)] @ self.E(ts, c)
                                   for ts in (tr.son0[t], tr.son1[t])])
                self.R[P.tc(t, c)] = qr_r(a, self.k)

    # -- step 2 ----------------------------------------------------------------
    def block_norms(self):
        P = self.pairs
        adm = self.dh2.blocks.adm
        self.bnorm = np.zeros(len(adm))
        for b, (t, s, c) in enumerate(adm):
            g = self.R[P.tc(t, c)] @ self.S(b) @ self.R[P.tc(s, c)].conj().T
            self.bnorm[b] = np.linalg.norm(g)

    # -- step 3 ----------------------------------------------------------------
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
                        parts.append(self.R[P.tc(sb, c)] @ self.S(b).conj().T / self.bnorm[b])
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

    # -- step 4 ----------------------------------------------------------------
    def truncate(self, Z):
        tr, P, d = self.tree, self.pairs, self.dh2
        Q, F, C, sig, rank = {}, {}, {}, {}, {}
        for l in range(tr.depth, -1, -1):
            for t, c in self.active_pairs(l):
                tc = P.tc(t, c)
                if tr.is_leaf(t):
                    V = d.leaf_basis(t, c)
                else:
                    c1 = d.son_direction(t, c)
                    V = np.vstack([C[P.tc(ts, c1)] @ self.E(ts, c)
                                   for ts in (tr.son0[t], tr.son1[t])])
                A = V @ Z[tc].conj().T
                if min(A.shape) == 0:
                    U = np.zeros((A.shape[0], 0), dtype=np.complex128)
                    s = np.zeros(0)
                else:
                    U, s, _ = np.linalg.svd(A, full_matrices=False)
                kk = choose_rank(s, self.eps, self.rule)
                Qt = U[:, :kk]
                sig[tc] = s
                rank[tc] = kk
                C[tc] = Qt.conj().T @ V
                if tr.is_leaf(t):
                    Q[tc] = Qt
                else:
                    k1 = C[P.tc(tr.son0[t], c1)].shape[0]
                    F[P.tc(tr.son0[t], c1), tc] = Qt[:k1]
                    F[P.tc(tr.son1[t], c1), tc] = Qt[k1:]
                    Q[tc] = Qt           # Q-hat for non-leaves
        return {"Q": Q, "F": F, "C": C, "sigma": sig, "rank": rank}

    def transfer_new(self, basis, tson, tc_parent, c_son):
        return basis["F"][self.pairs.tc(tson, c_son), tc_parent]

    # -- step 5 ----------------------------------------------------------------
    def project(self):
        P = self.pairs
        self.Stilde = []
        for b, (t, s, c) in enumerate(self.dh2.blocks.adm):
            self.Stilde.append(self.row["C"][P.tc(t, c)] @ self.S(b)
                               @ self.col["C"][P.tc(s, c)].conj().T)

    # -- expanded bases (tests) ------------------------------------------------
    def full_new_basis(self, basis, t, c):
        """Q_tc expanded to (#t, k_tc) through the new transfers F."""
        tr, P, d = self.tree, self.pairs, self.dh2
        tc = P.tc(t, c)
        if tr.is_leaf(t):
            return basis["Q"][tc]
        c1 = d.son_direction(t, c)
        return np.vstack([self.full_new_basis(basis, ts, c1) @ basis["F"][P.tc(ts, c1), tc]
                          for ts in (tr.son0[t], tr.son1[t])])

    def to_dense(self):
        """Expanded recompressed matrix in original numbering (tiny meshes)."""
        tr, P, d = self.tree, self.pairs, self.dh2
        n = tr.n
        A = np.zeros((n, n), dtype=np.complex128)
        for (t, s) in d.blocks.near:
            A[np.ix_(tr.indices(t), tr.indices(s))] = d.nearfield_block(t, s)
        for b, (t, s, c) in enumerate(d.blocks.adm):
            A[np.ix_(tr.indices(t), tr.indices(s))] = (
                self.full_new_basis(self.row, t, c) @ self.Stilde[b]
                @ self.full_new_basis(self.col, s, c).conj().T)
        return A

    # -- step 6 ----------------------------------------------------------------
    def matvec(self, x, near_blocks=None):
        """y = G~ x with the recompressed DH^2 matrix (x, y in original numbering)."""
        tr, P, d = self.tree, self.pairs, self.dh2
        xt = x[tr.perm]
        yt = np.zeros(tr.n, dtype=np.complex128)
        # forward transform (column basis), bottom-up
        xh = {}
        for l in range(tr.depth, -1, -1):
            for s, c in self.active_pairs(l):
                sc = P.tc(s, c)
                if tr.is_leaf(s):
                    o = tr.offset[s]
                    xh[sc] = self.col["Q"][sc].conj().T @ xt[o:o + tr.size[s]]
                else:
                    c1 = d.son_direction(s, c)
                    acc = np.zeros(self.col["rank"][sc], dtype=np.complex128)
                    for ss in (tr.son0[s], tr.son1[s]):
                        acc += self.col["F"][P.tc(ss, c1), sc].conj().T @ xh[P.tc(ss, c1)]
                    xh[sc] = acc
        # couplings
        yh = {}
        for l in range(tr.depth + 1):
            for t, c in self.active_pairs(l):
                tc = P.tc(t, c)
                acc = np.zeros(self.row["rank"][tc], dtype=np.complex128)
                for b in P.row[tc]:
                    s = d.blocks.adm[b][1]
                    acc += self.Stilde[b] @ xh[P.tc(s, c)]
                yh[tc] = acc
        # backward transform (row basis), top-down
        for l in range(tr.depth + 1):
            for t, c in self.active_pairs(l):
                tc = P.tc(t, c)
                if tr.is_leaf(t):
                    o = tr.offset[t]
                    yt[o:o + tr.size[t]] += self.row["Q"][tc] @ yh[tc]
                else:
                    c1 = d.son_direction(t, c)
                    for ts in (tr.son0[t], tr.son1[t]):
                        yh[P.tc(ts, c1)] = yh[P.tc(ts, c1)] + self.row["F"][P.tc(ts, c1), tc] @ yh[tc]
        # nearfield
        near = d.blocks.near if near_blocks is None else near_blocks
        for (t, s) in near:
            ot, os_ = tr.offset[t], tr.offset[s]
            yt[ot:ot + tr.size[t]] += d.nearfield_block(t, s) @ xt[os_:os_ + tr.size[s]]
        y = np.empty_like(yt)
        y[tr.perm] = yt
        return y
