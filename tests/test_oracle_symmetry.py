"""Pins of the complex symmetry that the GPU build uses to derive its column pass.

The Galerkin matrix of Eq. 2 is complex symmetric, G^T = G: g(x, y) = g(y, x) (Eq. 1) and
the same piecewise-constant basis functions stand on both sides.  The direction sets of
the Remark "construction of directions" are point-symmetric, D_l = -D_l, so the block
tree pairs every admissible block (t, s, c) with (s, t, -c), and W = V with
V_{t,-c} = conj(V_{t,c}).  Then the column-pass total weight of (t, c) has the Gram matrix
of the conjugated row-pass total weight of (t, -c), the two truncations have the same
singular values and ranks, and the basis weights of (t, -c) are the conjugates of those
of (t, c).  These tests check each fact on the oracle, which computes both passes
independently, and on the structure of every test case.
"""
import functools

import numpy as np
import pytest

from oracle.geometry import Discretisation
from oracle.interp import InterpolatedDH2
from oracle.recompress import Recompression
from oracle.structure import PairIndex, build_block_tree, build_cluster_tree, build_directions
from tests.cases import CASES, mesh, params


@functools.lru_cache(maxsize=None)
def _structure(name):
    v, f = mesh(name)
    p = params(name)
    tr = build_cluster_tree(v, f, p["leaf"])
    dirs = build_directions(tr, p["kappa"], p["eta1"])
    bt = build_block_tree(tr, dirs, p["kappa"], p["eta2"])
    return v, f, p, tr, dirs, bt


def _mirror(dirs, level):
    """Index of -c in D_level for every c (to 1e-12), or None where there is none."""
    D = np.asarray(dirs.dirs[level])
    out = []
    for c in range(len(D)):
        d = np.abs(D + D[c]).max(axis=1)
        j = int(np.argmin(d))
        out.append(j if d[j] <= 1e-12 else None)
    return out


def _symmetric_on_active_pairs(tr, dirs, bt):
    """The conditions of the mirrored column pass: every active pair (t, c) has an active
    mirror (t, -c) whose sons are the mirrors of its sons, and every admissible block
    (t, s, c) has its transpose (s, t, -c)."""
    mirrors = [_mirror(dirs, l) for l in range(tr.depth + 1)]
    P = PairIndex(tr, dirs, bt)
    for t in range(tr.nc):
        l = tr.level[t]
        for c in range(P.count[t]):
            if not P.active[P.base[t] + c]:
                continue
            cm = mirrors[l][c]
            if cm is None or not P.active[P.base[t] + cm]:
                return False
            if not tr.is_leaf(t) and dirs.sd[l][cm] != mirrors[l + 1][dirs.sd[l][c]]:
                return False
    blocks = {(int(t), int(s), int(c)) for t, s, c in bt.adm}
    for t, s, c in blocks:
        cm = mirrors[tr.level[t]][c]
        if cm is None or (s, t, cm) not in blocks:
            return False
    return True


def test_direction_sets_are_point_symmetric():
    """D_l = -D_l on every level of every case (to 1e-12), and the mirror is an involution."""
    for name in CASES:
        if name == "plain5120m5":
            continue
        _, _, _, tr, dirs, _ = _structure(name)
        for l in range(tr.depth + 1):
            mr = _mirror(dirs, l)
            assert all(j is not None for j in mr), (name, l)
            assert all(mr[j] == c for c, j in enumerate(mr)), (name, l)


def test_block_trees_without_directional_blocks_are_symmetric():
    """Where every admissible block lies on a level with D_l = {0} the mirror conditions
    hold exactly; the directional cases break them only by ties of the nearest-direction
    rules (sd and c_ts, ties to the lowest index), which the GPU build detects."""
    expect = {"laplace1280": True, "lowfreq1280": True, "plain1280": True, "dir320": False, "dir1280": False}
    for name, want in expect.items():
        _, _, _, tr, dirs, bt = _structure(name)
        assert _symmetric_on_active_pairs(tr, dirs, bt) == want, name


@pytest.mark.parametrize("name", ["laplace1280", "lowfreq1280"])
def test_column_pass_is_the_conjugated_row_pass(name):
    v, f, p, tr, dirs, bt = _structure(name)
    d = InterpolatedDH2(Discretisation(v, f), tr, dirs, bt, p["kappa"], p["m"])
    rc = Recompression(d, p["eps"])
    P = rc.pairs
    mirrors = [_mirror(dirs, l) for l in range(tr.depth + 1)]
    # the interpolated leaf bases and couplings: V_{t,-c} = conj(V_{t,c}), S_(s,t,-c) = S_(t,s,c)^T
    index = {(int(t), int(s), int(c)): b for b, (t, s, c) in enumerate(bt.adm)}
    for (t, s, c), b in list(index.items())[:50]:
        b2 = index[(s, t, mirrors[tr.level[t]][c])]
        S, S2 = rc.S(b), rc.S(b2)
        assert np.abs(S2 - S.T).max() <= 1e-12 * np.abs(S).max()
    checked = 0
    for l in range(tr.depth + 1):
        for t, c in rc.active_pairs(l):
            tc, tm = P.tc(t, c), P.tc(t, mirrors[l][c])
            if tr.is_leaf(t):
                V, Vm = d.leaf_basis(t, c), d.leaf_basis(t, mirrors[l][c])
                assert np.abs(Vm - V.conj()).max() <= 1e-12 * max(np.abs(V).max(), 1e-300)
            R, Rm = rc.R[tc], rc.R[tm]
            g, gm = R.conj().T @ R, Rm.conj().T @ Rm
            assert np.linalg.norm(gm - g.conj()) <= 1e-10 * max(np.linalg.norm(g), 1e-300)
            zc, zr = rc.ZC[tc], rc.ZR[tm]
            gc, gr = zc.conj().T @ zc, zr.conj().T @ zr
            assert np.linalg.norm(gc - gr.conj()) <= 1e-10 * max(np.linalg.norm(gr), 1e-300), (t, c)
            sc, sr = rc.col["sigma"][tc], rc.row["sigma"][tm]
            n = min(len(sc), len(sr))
            if n:
                assert np.abs(sc[:n] ** 2 - sr[:n] ** 2).max() <= 1e-10 * sr[0] ** 2
            assert rc.col["rank"][tc] == rc.row["rank"][tm]
            checked += 1
    assert checked > 0
