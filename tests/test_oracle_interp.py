"""Pins of the oracle's directional interpolation (Section 2: Lagrange polynomials,
Eq. matrix_apx, Eq. nested_apx, Eq. nested)."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev

from oracle.geometry import Discretisation
from oracle.interp import ChebyshevBoxes, InterpolatedDH2
from oracle.structure import build_block_tree, build_cluster_tree, build_directions
from tests.cases import mesh, params


def _dh2(name, m=None, kappa=None):
    v, f = mesh(name)
    p = params(name)
    if kappa is not None:
        p["kappa"] = kappa
    tr = build_cluster_tree(v, f, p["leaf"])
    dirs = build_directions(tr, p["kappa"], p["eta1"])
    bt = build_block_tree(tr, dirs, p["kappa"], p["eta2"])
    return InterpolatedDH2(Discretisation(v, f), tr, dirs, bt, p["kappa"], m or p["m"]), p


@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_nodes_are_chebyshev_roots_and_lagrange_is_delta(m):
    d, _ = _dh2("dir320", m=m)
    cb = d.cheb
    t = 5
    for axis in range(3):
        lo, hi = d.tree.lo[t, axis], d.tree.hi[t, axis]
        half = max((hi - lo) / 2, 1e-3 * ((d.tree.hi[t] - d.tree.lo[t]) / 2).max())
        ref = (cb.nodes[t, axis] - (lo + hi) / 2) / half
        # roots of T_m
        assert np.allclose(chebyshev.chebval(ref, [0] * m + [1]), 0.0, atol=1e-12)
        assert len(np.unique(np.round(ref, 12))) == m
        L = cb.lagrange_1d(t, axis, cb.nodes[t, axis])
        assert np.allclose(L, np.eye(m), atol=1e-13)


@pytest.mark.parametrize("m", [2, 3, 4])
def test_interpolation_reproduces_tensor_polynomials(m):
    d, _ = _dh2("dir320", m=m)
    t = 3
    xi = d.cheb.points(t)
    rng = np.random.default_rng(5)
    x = d.tree.lo[t] + rng.random((40, 3)) * (d.tree.hi[t] - d.tree.lo[t])
    L = d.cheb.lagrange(t, x)
    for a in range(m):
        for b in range(m):
            for c in range(m):
                p = lambda z: z[:, 0] ** a * z[:, 1] ** b * z[:, 2] ** c
                assert np.allclose(L @ p(xi), p(x), rtol=1e-10, atol=1e-12)
    # degree m in one variable is not reproduced (the pin can fail)
    p = lambda z: z[:, 0] ** m
    assert np.abs(L @ p(xi) - p(x)).max() > 1e-8 * np.abs(p(x)).max()


def test_leaf_basis_integrates_quadratics_exactly():
    """With c = 0 and m >= 3, sum_nu V_{i nu} p(xi_nu) = int_{T_i} p for total degree <= 2."""
    d, _ = _dh2("lowfreq1280", m=3)
    disc = d.disc
    leaves = [t for t in range(d.tree.nc) if d.tree.is_leaf(t)][:5]
    for t in leaves:
        V = d.leaf_basis(t, 0)
        xi = d.cheb.points(t)
        idx = d.tree.indices(t)
        verts = disc.vertices[disc.triangles[idx]]        # (#t, 3, 3)
        area = disc.area[idx]
        cen = verts.mean(1)
        # int_T x = |T| centroid_x ; int_T x^2 = |T|/12 (sum v_i^2 + (sum v_i)^2)
        assert np.allclose(V @ xi[:, 0], area * cen[:, 0], rtol=1e-11, atol=1e-14)
        assert np.allclose(V @ np.ones(len(xi)), area, rtol=1e-12)
        sq = area / 12.0 * ((verts[:, :, 1] ** 2).sum(1) + verts[:, :, 1].sum(1) ** 2)
        assert np.allclose(V @ xi[:, 1] ** 2, sq, rtol=1e-10, atol=1e-14)
        xy = area / 12.0 * ((verts[:, :, 0] * verts[:, :, 2]).sum(1)
                            + verts[:, :, 0].sum(1) * verts[:, :, 2].sum(1))
        assert np.allclose(V @ (xi[:, 0] * xi[:, 2]), xy, rtol=1e-10, atol=1e-14)


def test_nested_exact_without_directions():
    """c = c' = 0: V_t restricted to t' equals V_{t'} E_{t'} (polynomial reproduction)."""
    d, _ = _dh2("lowfreq1280", m=3)
    tr = d.tree
    checked = 0
    for t in range(tr.nc):
        if tr.is_leaf(t) or not (tr.is_leaf(tr.son0[t]) and tr.is_leaf(tr.son1[t])):
            continue
        Vt = np.vstack([d.leaf_basis(ts, 0) @ d.transfer(ts, 0) for ts in (tr.son0[t], tr.son1[t])])
        # direct evaluation of the father's Lagrange polynomials on the sons' triangles
        idx = tr.indices(t)
        x = d.disc.x3[idx].reshape(-1, 3)
        direct = np.einsum("iq,iqn->in", d.disc.w3[idx], d.cheb.lagrange(t, x).reshape(len(idx), 3, -1))
        assert np.allclose(Vt, direct, rtol=1e-10, atol=1e-13 * np.abs(direct).max())
        checked += 1
        if checked > 4:
            break
    assert checked > 0


def test_nested_error_linear_in_phase_mismatch():
    """c != 0: Eq. (nested_apx) interpolates exp(i kappa <x, c - c'>) L_t on B_t'.  Its
    error is first order in kappa |c - c'| diam(B_t') (the Lagrange polynomial times the
    linear term of the plane wave leaves the polynomial space), so with the directions
    held fixed it scales linearly with kappa, and vanishes for kappa -> 0."""
    base, p = _dh2("dir320", m=4)
    tr, dirs = base.tree, base.dirs
    t = next(t for t in range(tr.nc) if not tr.is_leaf(t) and dirs.msplit[tr.level[t]] > 0
             and tr.is_leaf(tr.son0[t]) and tr.is_leaf(tr.son1[t]))
    errs = []
    for scale in (1.0, 0.1, 0.01):
        d = InterpolatedDH2(base.disc, tr, dirs, base.blocks, p["kappa"] * scale, 4)
        c = 3
        idx = tr.indices(t)
        x = d.disc.x3[idx].reshape(-1, 3)
        wave = np.exp(1j * d.kappa * (x @ dirs.dirs[tr.level[t]][c]))
        lag = d.cheb.lagrange(t, x) * wave[:, None]
        direct = np.einsum("iq,iqn->in", d.disc.w3[idx], lag.reshape(len(idx), 3, -1))
        c1 = dirs.sd[tr.level[t]][c]
        nested = np.vstack([d.leaf_basis(ts, c1) @ d.transfer(ts, c) for ts in (tr.son0[t], tr.son1[t])])
        errs.append(np.linalg.norm(nested - direct) / np.linalg.norm(direct))
    assert 5.0 < errs[0] / errs[1] < 20.0
    assert 5.0 < errs[1] / errs[2] < 20.0
    assert errs[0] < 0.05


def test_coupling_is_plane_wave_split_kernel():
    d, _ = _dh2("dir320")
    b = 0
    t, s, c = d.blocks.adm[b]
    S = d.coupling(b)
    xt, xs = d.cheb.points(t), d.cheb.points(s)
    cv = d.direction(t, c)
    diff = xt[:, None, :] - xs[None, :, :]
    r = np.linalg.norm(diff, axis=2)
    g = np.exp(1j * d.kappa * r) / (4 * math.pi * r)
    assert np.allclose(S * np.exp(1j * d.kappa * (diff @ cv)), g, rtol=1e-12)


def test_interpolated_matrix_converges_to_dense():
    """Interpolation error of the analytic DH^2 matrix falls with m (convergence, reported)."""
    errs = []
    for m in (2, 3, 4):
        d, p = _dh2("dir320", m=m)
        G = d.disc.dense(p["kappa"])
        A = d.to_dense()
        errs.append(np.linalg.norm(A - G) / np.linalg.norm(G))
        x = np.random.default_rng(1).standard_normal(d.tree.n) + 0j
        assert np.allclose(d.matvec(x), A @ x, rtol=1e-12, atol=1e-14)
    assert errs[2] < errs[0] * 0.2
