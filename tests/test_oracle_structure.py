"""Pins of the oracle's cluster tree, directions and block tree (Defs. cluster tree,
directions, block tree; Eq. 3, Eq. 4; Remark "construction of directions")."""
import math

import numpy as np
import pytest

import synth
from oracle.structure import (build_block_tree, build_cluster_tree, build_directions,
                              centroids, PairIndex, point_cluster_tree)
from tests.cases import mesh, params


def _tree(name):
    v, f = mesh(name)
    p = params(name)
    return v, f, build_cluster_tree(v, f, p["leaf"]), p


@pytest.mark.parametrize("name", ["plain1280", "dir1280", "dir320"])
def test_cluster_tree_partition(name):
    v, f, tr, p = _tree(name)
    n = len(f)
    assert sorted(tr.perm.tolist()) == list(range(n))
    assert tr.offset[0] == 0 and tr.size[0] == n and tr.level[0] == 0
    cent = centroids(v, f)
    tv = v[f]
    for t in range(tr.nc):
        idx = tr.indices(t)
        # boxes contain the triangles and are tight
        assert np.all(tv[idx].min(axis=(0, 1)) == tr.lo[t])
        assert np.all(tv[idx].max(axis=(0, 1)) == tr.hi[t])
        if tr.is_leaf(t):
            assert tr.size[t] <= p["leaf"]
            continue
        assert tr.size[t] > p["leaf"]
        s0, s1 = tr.son0[t], tr.son1[t]
        assert tr.parent[s0] == t and tr.parent[s1] == t
        assert tr.level[s0] == tr.level[t] + 1 == tr.level[s1]
        # sons partition the father, contiguous, left first
        assert tr.offset[s0] == tr.offset[t]
        assert tr.offset[s1] == tr.offset[t] + tr.size[s0]
        assert tr.size[s0] + tr.size[s1] == tr.size[t]
        assert tr.size[s0] > 0 and tr.size[s1] > 0
        # the split separates the centroids along the longest centroid-box axis
        c = cent[idx]
        ext = c.max(0) - c.min(0)
        axis = int(np.argmax(ext))
        split = (c[:, axis].min() + c[:, axis].max()) * 0.5
        assert np.all(cent[tr.indices(s0), axis] < split)
        assert np.all(cent[tr.indices(s1), axis] >= split)
        # stability: relative order of the original indices is kept on each side
        for s in (s0, s1):
            sub = tr.indices(s)
            pos = {int(x): i for i, x in enumerate(idx)}
            assert all(pos[int(a)] < pos[int(b)] for a, b in zip(sub[:-1], sub[1:]))
    # levels are numbered contiguously, breadth first
    assert np.all(np.diff(tr.level) >= 0)


def test_cluster_tree_median_fallback():
    """Identical centroids along the split axis force the median rule."""
    pts = np.zeros((10, 3))
    pts[:, 1] = np.arange(10) * 0.0
    tr = point_cluster_tree(pts, leaf_max=4)
    assert tr.size[tr.son0[0]] == 5 and tr.size[tr.son1[0]] == 5
    assert tr.indices(tr.son0[0]).tolist() == [0, 1, 2, 3, 4]


def test_direction_family_covering():
    """|D_l| = 6 m_l^2 unit vectors covering the sphere within eta1/(kappa d_l) (Eq. 4)."""
    v, f, tr, p = _tree("dir1280")
    dirs = build_directions(tr, p["kappa"], p["eta1"])
    rng = np.random.default_rng(11)
    y = rng.standard_normal((4000, 3))
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    nonzero_levels = 0
    for l in range(tr.depth + 1):
        D = dirs.dirs[l]
        if dirs.msplit[l] == 0:
            assert D.shape == (1, 3) and np.all(D == 0)
            assert p["kappa"] * dirs.dmax[l] <= p["eta1"]
            continue
        nonzero_levels += 1
        m = dirs.msplit[l]
        assert len(D) == 6 * m * m
        assert m == math.ceil(math.sqrt(2) * p["kappa"] * dirs.dmax[l] / p["eta1"])
        assert np.allclose(np.linalg.norm(D, axis=1), 1.0, atol=1e-15)
        # closed under c -> -c (the face grid is symmetric)
        assert np.allclose(np.sort(D, axis=0), np.sort(-D, axis=0))
        dist = np.sqrt(((y[:, None, :] - D[None, :, :]) ** 2).sum(-1)).min(1)
        assert dist.max() <= p["eta1"] / (p["kappa"] * dirs.dmax[l]) + 1e-12
        assert dist.max() <= math.sqrt(2) / m + 1e-12
    assert nonzero_levels >= 3


def test_son_map_is_nearest():
    v, f, tr, p = _tree("dir1280")
    dirs = build_directions(tr, p["kappa"], p["eta1"])
    for l in range(tr.depth):
        D0, D1 = dirs.dirs[l], dirs.dirs[l + 1]
        d2 = ((D0[:, None, :] - D1[None, :, :]) ** 2).sum(-1)
        best = d2.min(1)
        got = d2[np.arange(len(D0)), dirs.sd[l]]
        assert np.allclose(got, best, rtol=0, atol=1e-15)


@pytest.mark.parametrize("name", ["laplace1280", "lowfreq1280", "dir1280", "dir320", "plain1280"])
def test_block_tree_partition_and_admissibility(name):
    v, f, tr, p = _tree(name)
    dirs = build_directions(tr, p["kappa"], p["eta1"])
    bt = build_block_tree(tr, dirs, p["kappa"], p["eta2"])
    n = tr.n
    cover = np.zeros((n, n), dtype=np.int8)
    diam = np.linalg.norm(tr.hi - tr.lo, axis=1)
    mid = tr.mid()

    def dist(t, s):
        gap = np.maximum(0.0, np.maximum(tr.lo[t] - tr.hi[s], tr.lo[s] - tr.hi[t]))
        return np.linalg.norm(gap)

    def adm(t, s):
        dd = dist(t, s)
        return (max(diam[t], diam[s]) <= p["eta2"] * dd
                and p["kappa"] * max(diam[t], diam[s]) ** 2 <= p["eta2"] * dd)

    for (t, s, c) in bt.adm:
        assert tr.level[t] == tr.level[s]
        assert adm(t, s)
        if t != 0:
            assert not adm(tr.parent[t], tr.parent[s])
        cover[np.ix_(tr.indices(t), tr.indices(s))] += 1
        # c_ts is a best approximation of (m_t - m_s)/|m_t - m_s|
        D = dirs.dirs[tr.level[t]]
        if len(D) > 1:
            u = (mid[t] - mid[s])
            u = u / np.linalg.norm(u)
            d2 = ((D - u) ** 2).sum(1)
            assert d2[c] <= d2.min() + 1e-15
            # Eq. (3a) then holds by Eq. (4)
            assert p["kappa"] * np.linalg.norm(u - D[c]) <= p["eta1"] / max(diam[t], diam[s]) + 1e-12
    for (t, s) in bt.near:
        assert tr.level[t] == tr.level[s]
        assert not adm(t, s)
        assert tr.is_leaf(t) or tr.is_leaf(s)
        if t != 0:
            assert not adm(tr.parent[t], tr.parent[s])
        cover[np.ix_(tr.indices(t), tr.indices(s))] += 1
    assert np.all(cover == 1)


def test_structure_counts_cross_check():
    """Counts agree with an independent throwaway implementation of the same readings
    (1280-triangle icosphere): C1 has no admissible block; the stress sets do."""
    v, f = synth.icosphere(3)
    expect = {(4.0, 32, 10.0, 1.0): (103, 6, 0, 2224), (0.0, 32, 10.0, 1.0): (103, 6, 794, None),
              (4.0, 16, 10.0, 1.0): (221, 8, 272, None), (8.0, 8, 1.0, 2.0): (433, 9, 16248, None)}
    for (kappa, leaf, eta1, eta2), (nc, depth, na, nn) in expect.items():
        tr = build_cluster_tree(v, f, leaf)
        dirs = build_directions(tr, kappa, eta1)
        bt = build_block_tree(tr, dirs, kappa, eta2)
        assert (tr.nc, tr.depth, len(bt.adm)) == (nc, depth, na)
        if nn is not None:
            assert len(bt.near) == nn


def test_active_pairs_closed_downward():
    v, f, tr, p = _tree("dir1280")
    dirs = build_directions(tr, p["kappa"], p["eta1"])
    bt = build_block_tree(tr, dirs, p["kappa"], p["eta2"])
    P = PairIndex(tr, dirs, bt)
    for t in range(tr.nc):
        for c in range(P.count[t]):
            if P.active[P.tc(t, c)] and not tr.is_leaf(t):
                c1 = dirs.sd[tr.level[t]][c]
                assert P.active[P.tc(tr.son0[t], c1)] and P.active[P.tc(tr.son1[t], c1)]
    for b, (t, s, c) in enumerate(bt.adm):
        assert b in P.row[P.tc(t, c)] and b in P.col[P.tc(s, c)]
