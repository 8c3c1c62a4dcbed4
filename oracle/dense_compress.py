"""Section 3.1 compression applied to an explicitly assembled matrix (oracle, tiny meshes).

Test infrastructure only (see ``oracle/__init__``).

For a pair (t,c) the paper collects every admissible block of the ancestors
anc(t,c) (Eq. ancestors) in G_tc = G|_{t x R_tc}.  Here G is the interpolated
DH^2 matrix and every block enters with the same weight 1/||G_b||_F as in the
fast algorithm.  For a leaf the left singular values of G_tc decide the rank;
for a non-leaf the same holds for G-hat_tc = diag(Q_{t1c1}^*, Q_{t2c2}^*) G_tc
(Eq. Ghat) with the sons' new bases.  The paper states that the factorisation
G_tc = V_tc Z-hat_tc^* P_tc^* (Eq. recomp_weight_full) leaves these singular
values unchanged; the tests use this as a brute-force pin of Section 3.2.
"""
from __future__ import annotations

import numpy as np

from .recompress import Recompression


def ancestors(rc: Recompression, t, c):
    """anc(t,c) of Eq. (ancestors) as a list of (t~, c~)."""
    tr, P = rc.tree, rc.pairs
    out = [(int(t), int(c))]
    tp = tr.parent[t]
    if tp >= 0:
        for cp in P.sd_inverse(tp, c):
            out += ancestors(rc, tp, cp)
    return out


def explicit_Gtc(rc: Recompression, t, c, rows=True):
    """Weighted G_tc assembled block by block from the interpolated matrix."""
    tr, P, d = rc.tree, rc.pairs, rc.dh2
    o, n_t = tr.offset[t], tr.size[t]
    cols = []
    for (ta, ca) in ancestors(rc, t, c):
        tca = P.tc(ta, ca)
        for b in (P.row[tca] if rows else P.col[tca]):
            tb, sb, cb = d.blocks.adm[b]
            Vt = d.full_basis(tb, cb)
            Vs = d.full_basis(sb, cb)
            blk = Vt @ rc.S(b) @ Vs.conj().T / rc.bnorm[b]
            if not rows:
                blk = blk.conj().T          # G^* restricted to s x t
            cols.append(blk[o - tr.offset[ta]: o - tr.offset[ta] + n_t])
    if not cols:
        return np.zeros((n_t, 0), dtype=np.complex128)
    return np.hstack(cols)


def dense_singular_values(rc: Recompression, t, c, rows=True):
    """Singular values of G_tc (leaf) or G-hat_tc (non-leaf), Section 3.1."""
    tr, P, d = rc.tree, rc.pairs, rc.dh2
    G = explicit_Gtc(rc, t, c, rows)
    basis = rc.row if rows else rc.col
    if not tr.is_leaf(t):
        c1 = d.son_direction(t, c)
        blocks = []
        o = tr.offset[t]
        for ts in (tr.son0[t], tr.son1[t]):
            Qs = rc.full_new_basis(basis, ts, c1)
            r0 = tr.offset[ts] - o
            blocks.append(Qs.conj().T @ G[r0:r0 + tr.size[ts]])
        G = np.vstack(blocks)
    if min(G.shape) == 0:
        return np.zeros(0)
    return np.linalg.svd(G, compute_uv=False)
