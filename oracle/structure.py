"""Cluster tree, bounding boxes, directions and block tree (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).  Everything here decides
integers (splits, levels, directions, block types) from FP64 values, so each
formula is written with an explicit evaluation order; the CUDA path evaluates
the same expressions with round-to-nearest and no contraction, and parity is
bit-exact.

Readings where the paper is silent (Section 5 only says "standard binary space
partitioning until clusters contain not more than 32 elements"):

* split along the longest axis of the cluster's *centroid* box (ties -> lowest
  axis) at (lo + hi) * 0.5; element goes left iff centroid[axis] < split;
  stable partition, left child first; if one side would be empty, the first
  floor(size/2) elements in (centroid[axis], index) order go left;
* a cluster is a leaf iff size <= leaf_max; clusters are numbered level by
  level (children appended in the order their parents are visited);
* B_t = vertex box of the cluster's triangles (so supp phi_i lies in B_t,
  Section 2); diam = Euclidean diagonal, dist = Euclidean box gap, m_t = box
  centre;
* centroid = ((v0 + v1) + v2) / 3.

Directions (Remark "construction of directions"): d_l = max diam on level l;
D_l = {0} iff kappa d_l <= eta1; otherwise m_l = ceil(sqrt(2) kappa d_l / eta1)
and the 6 m_l^2 face centres of the cube [-1,1]^3 (the paper's "[0,1]^3"
contradicts its own square width 2/m) projected to the sphere, faces ordered
(+x,-x,+y,-y,+z,-z), first free axis outer.  sd_l(c) = nearest direction on
level l+1 (Def. "directions"), ties to the lowest index.  c_ts = best
approximation of (m_t - m_s)/|m_t - m_s| (Section 2), ties lowest, index 0 if
m_t = m_s.

Block tree (Def. "block tree"): a pair is an admissible leaf iff it satisfies
(3b) max(diam) <= eta2 dist and (3c) kappa max(diam^2) <= eta2 dist; (3a)
then holds for c_ts by Eq. (4).  Otherwise, if both clusters have sons, the
four son pairs follow in (t-son, s-son) order; else it is a nearfield leaf.
The recursion is breadth first, level by level.

Pins (tests/test_oracle_structure.py): partition invariants of the cluster tree
(Def. "cluster tree"); the block leaves partition I x I; admissible leaves
satisfy (3b)/(3c) and their parents do not; level(t) = level(s); |D_l| = 6 m_l^2
unit vectors; the covering bound Eq. (4) on random unit vectors; sd and c_ts
are nearest by brute force.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class ClusterTree:
    n: int
    leaf_max: int
    perm: np.ndarray            # perm[i] = original index of the i-th element in cluster order
    offset: np.ndarray          # per cluster
    size: np.ndarray
    parent: np.ndarray          # -1 for the root
    son0: np.ndarray            # -1 for leaves
    son1: np.ndarray
    level: np.ndarray
    lo: np.ndarray              # (nc, 3) vertex box
    hi: np.ndarray
    level_start: np.ndarray     # clusters of level l are level_start[l]:level_start[l+1]

    @property
    def nc(self):
        return len(self.offset)

    @property
    def depth(self):
        return len(self.level_start) - 2

    def is_leaf(self, t):
        return self.son0[t] < 0

    def indices(self, t):
        return self.perm[self.offset[t]:self.offset[t] + self.size[t]]

    def diam(self):
        d = self.hi - self.lo
        return np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])

    def mid(self):
        return (self.lo + self.hi) * 0.5


def centroids(vertices, triangles):
    v0, v1, v2 = (vertices[triangles[:, j]] for j in range(3))
    return ((v0 + v1) + v2) / 3.0


def build_cluster_tree(vertices, triangles, leaf_max=32):
    """Binary space partitioning cluster tree (Def. "cluster tree", Section 5)."""
    vertices = np.asarray(vertices, dtype=np.float64)
    triangles = np.asarray(triangles, dtype=np.int64)
    n = len(triangles)
    cent = centroids(vertices, triangles)
    tv = vertices[triangles]                      # (n, 3 vertices, 3)
    tlo = np.minimum(np.minimum(tv[:, 0], tv[:, 1]), tv[:, 2])
    thi = np.maximum(np.maximum(tv[:, 0], tv[:, 1]), tv[:, 2])

    perm = np.arange(n, dtype=np.int64)
    offset, size, parent, son0, son1, level = [0], [n], [-1], [], [], [0]
    lo, hi = [], []
    t = 0
    while t < len(offset):
        off, sz = offset[t], size[t]
        idx = perm[off:off + sz]
        lo.append(tlo[idx].min(axis=0))
        hi.append(thi[idx].max(axis=0))
        if sz <= leaf_max:
            son0.append(-1)
            son1.append(-1)
        else:
            clo = cent[idx].min(axis=0)
            chi = cent[idx].max(axis=0)
            ext = chi - clo
            axis = 0
            for a in (1, 2):
                if ext[a] > ext[axis]:
                    axis = a
            split = (clo[axis] + chi[axis]) * 0.5
            key = cent[idx, axis]
            left = key < split
            nl = int(left.sum())
            if nl == 0 or nl == sz:
                order = np.lexsort((idx, key))          # by (key, original index)
                left = np.zeros(sz, dtype=bool)
                left[order[: sz // 2]] = True
                nl = sz // 2
            perm[off:off + sz] = np.concatenate([idx[left], idx[~left]])
            c0 = len(offset)
            for (o, s) in ((off, nl), (off + nl, sz - nl)):
                offset.append(o)
                size.append(s)
                parent.append(t)
                level.append(level[t] + 1)
            son0.append(c0)
            son1.append(c0 + 1)
        t += 1
    level = np.asarray(level, dtype=np.int64)
    nlev = int(level.max()) + 1
    level_start = np.searchsorted(level, np.arange(nlev + 1))
    return ClusterTree(
        n=n, leaf_max=leaf_max, perm=perm,
        offset=np.asarray(offset, dtype=np.int64), size=np.asarray(size, dtype=np.int64),
        parent=np.asarray(parent, dtype=np.int64), son0=np.asarray(son0, dtype=np.int64),
        son1=np.asarray(son1, dtype=np.int64), level=level,
        lo=np.asarray(lo), hi=np.asarray(hi), level_start=level_start,
    )


def point_cluster_tree(points, leaf_max=32):
    """Cluster tree for point elements (a degenerate triangle (p, p, p) per point)."""
    pts = np.asarray(points, dtype=np.float64)
    tri = np.repeat(np.arange(len(pts))[:, None], 3, axis=1)
    return build_cluster_tree(pts, tri, leaf_max)


# --------------------------------------------------------------------------- directions

@dataclass
class Directions:
    kappa: float
    eta1: float
    dmax: np.ndarray                                  # d_l per level
    msplit: np.ndarray                                # m_l per level (0 if D_l = {0})
    dirs: list = field(default_factory=list)          # dirs[l]: (|D_l|, 3)
    sd: list = field(default_factory=list)            # sd[l]: (|D_l|,) index into dirs[l+1]

    def count(self, l):
        return len(self.dirs[l])


def direction_set(msplit):
    """6 m^2 normalised face centres of [-1,1]^3 (Remark "construction of directions")."""
    out = []
    for axis in range(3):
        for sign in (1.0, -1.0):
            b, c = [a for a in range(3) if a != axis]
            for i in range(msplit):
                for j in range(msplit):
                    v = [0.0, 0.0, 0.0]
                    v[axis] = sign
                    v[b] = -1.0 + (2 * i + 1) / msplit
                    v[c] = -1.0 + (2 * j + 1) / msplit
                    nrm = math.sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2])
                    out.append([v[0] / nrm, v[1] / nrm, v[2] / nrm])
    return np.asarray(out, dtype=np.float64)


def nearest(u, cands):
    """Index of the candidate nearest to u, Euclidean, ties to the lowest index."""
    d = cands - u[None, :]
    dist2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    return int(np.argmin(dist2))          # argmin returns the first minimum


def nearest_many(us, cands, chunk=512):
    """``nearest`` for each row of ``us`` (same arithmetic, evaluated in chunks)."""
    out = np.empty(len(us), dtype=np.int64)
    for i0 in range(0, len(us), chunk):
        d = cands[None, :, :] - us[i0:i0 + chunk, None, :]
        dist2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        out[i0:i0 + chunk] = np.argmin(dist2, axis=1)
    return out


def build_directions(tree: ClusterTree, kappa, eta1=10.0):
    diam = tree.diam()
    nlev = tree.depth + 1
    dmax = np.array([diam[tree.level_start[l]:tree.level_start[l + 1]].max() for l in range(nlev)])
    msplit = np.zeros(nlev, dtype=np.int64)
    dirs = []
    for l in range(nlev):
        if kappa * dmax[l] <= eta1:
            dirs.append(np.zeros((1, 3)))
        else:
            m = int(math.ceil(math.sqrt(2.0) * kappa * dmax[l] / eta1))
            msplit[l] = m
            dirs.append(direction_set(m))
    sd = []
    for l in range(nlev - 1):
        sd.append(nearest_many(dirs[l], dirs[l + 1]))
    sd.append(np.zeros(len(dirs[-1]), dtype=np.int64))
    return Directions(kappa=kappa, eta1=eta1, dmax=dmax, msplit=msplit, dirs=dirs, sd=sd)


def block_direction(tree, dirs_l, t, s):
    """c_ts: best approximation of the direction from m_s to m_t (Section 2)."""
    if len(dirs_l) == 1:
        return 0
    mid = tree.mid()
    d = mid[t] - mid[s]
    nrm = math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
    if nrm == 0.0:
        return 0
    u = np.array([d[0] / nrm, d[1] / nrm, d[2] / nrm])
    return nearest(u, dirs_l)


# --------------------------------------------------------------------------- block tree

@dataclass
class BlockTree:
    adm: np.ndarray          # (na, 3): t, s, c (c = index into D_level(t)), breadth-first order
    near: np.ndarray         # (nn, 2): t, s, breadth-first order
    eta2: float


def box_dist(tree, t, s):
    g = np.maximum(np.maximum(tree.lo[t] - tree.hi[s], tree.lo[s] - tree.hi[t]), 0.0)
    return math.sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2])


def admissible(tree, diam, kappa, eta2, t, s):
    """Conditions (3b) and (3c) of Eq. (3)."""
    dist = box_dist(tree, t, s)
    dt, ds = float(diam[t]), float(diam[s])
    dmx = max(dt, ds)
    d2 = max(dt * dt, ds * ds)
    return dmx <= eta2 * dist and kappa * d2 <= eta2 * dist


def build_block_tree(tree: ClusterTree, dirs: Directions, kappa, eta2=1.0):
    diam = tree.diam()
    adm, near = [], []
    frontier = [(0, 0)]
    while frontier:
        nxt = []
        for (t, s) in frontier:
            if admissible(tree, diam, kappa, eta2, t, s):
                c = block_direction(tree, dirs.dirs[tree.level[t]], t, s)
                adm.append((t, s, c))
            elif not tree.is_leaf(t) and not tree.is_leaf(s):
                for tt in (tree.son0[t], tree.son1[t]):
                    for ss in (tree.son0[s], tree.son1[s]):
                        nxt.append((tt, ss))
            else:
                near.append((t, s))
        frontier = nxt
    return BlockTree(adm=np.asarray(adm, dtype=np.int64).reshape(-1, 3),
                     near=np.asarray(near, dtype=np.int64).reshape(-1, 2), eta2=eta2)


# --------------------------------------------------------------------------- (t,c) bookkeeping

class PairIndex:
    """Global enumeration of the pairs (t, c), c in D_level(t): tc = base[t] + c.

    row(t,c) / col(s,c) (Section 3.1) as lists of admissible block ids, sd^{-1},
    and the active set: pairs with a block in row or col, closed under
    (t, c) -> (t', sd(c)) for the sons t' (the pairs the recursions of
    Section 3.2 visit).  Lists are kept in block order.
    """

    def __init__(self, tree: ClusterTree, dirs: Directions, blocks: BlockTree):
        self.tree, self.dirs, self.blocks = tree, dirs, blocks
        cnt = np.array([dirs.count(tree.level[t]) for t in range(tree.nc)], dtype=np.int64)
        self.base = np.concatenate([[0], np.cumsum(cnt)])[:-1]
        self.count = cnt
        self.ntc = int(cnt.sum())
        self.row = [[] for _ in range(self.ntc)]
        self.col = [[] for _ in range(self.ntc)]
        for b, (t, s, c) in enumerate(blocks.adm):
            self.row[self.base[t] + c].append(b)
            self.col[self.base[s] + c].append(b)
        active = np.zeros(self.ntc, dtype=bool)
        for tc in range(self.ntc):
            active[tc] = bool(self.row[tc]) or bool(self.col[tc])
        for l in range(tree.depth + 1):
            for t in range(tree.level_start[l], tree.level_start[l + 1]):
                if tree.is_leaf(t):
                    continue
                for c in range(cnt[t]):
                    if active[self.base[t] + c]:
                        c1 = dirs.sd[l][c]
                        for tt in (tree.son0[t], tree.son1[t]):
                            active[self.base[tt] + c1] = True
        self.active = active

    def tc(self, t, c):
        return int(self.base[t] + c)

    def sd_inverse(self, t_parent, c_son):
        """Directions c+ of the parent with sd(c+) = c_son, ascending."""
        l = self.tree.level[t_parent]
        return [int(cp) for cp in np.nonzero(self.dirs.sd[l] == c_son)[0]]
