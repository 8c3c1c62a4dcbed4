"""Pins of the oracle's Section 3.2 recompression against Section 3.1 and closed forms."""
import functools
import math

import numpy as np
import pytest

import synth
from oracle.dense_compress import ancestors, dense_singular_values, explicit_Gtc
from oracle.geometry import Discretisation
from oracle.interp import InterpolatedDH2
from oracle.recompress import RANK_BLOCKREL, RANK_GLOBAL, RANK_SPECTRAL, Recompression, choose_rank
from oracle.structure import build_block_tree, build_cluster_tree, build_directions
from tests.cases import mesh, params


@functools.lru_cache(maxsize=None)
def _rc(name, eps=None, rule=RANK_BLOCKREL):
    v, f = mesh(name)
    p = params(name)
    tr = build_cluster_tree(v, f, p["leaf"])
    dirs = build_directions(tr, p["kappa"], p["eta1"])
    bt = build_block_tree(tr, dirs, p["kappa"], p["eta2"])
    d = InterpolatedDH2(Discretisation(v, f), tr, dirs, bt, p["kappa"], p["m"])
    return Recompression(d, eps or p["eps"], rule)


def _active(rc):
    P = rc.pairs
    for l in range(rc.tree.depth + 1):
        for t, c in rc.active_pairs(l):
            yield t, c, P.tc(t, c)


CASES = ["dir320", "mixed1280", "lowfreq1280"]


@pytest.mark.parametrize("name", CASES)
def test_basis_weights_gram(name):
    """R_tc^* R_tc = V_tc^* V_tc with V_tc expanded through Eq. (nested)."""
    rc = _rc(name)
    for t, c, tc in _active(rc):
        V = rc.dh2.full_basis(t, c)
        R = rc.R[tc]
        assert R.shape == (min(V.shape[0], rc.k) if rc.tree.is_leaf(t) else R.shape[0], rc.k)
        g = V.conj().T @ V
        assert np.linalg.norm(R.conj().T @ R - g) <= 1e-11 * np.linalg.norm(g)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("rows", [True, False])
def test_total_weights_factorise_Gtc(name, rows):
    """V_tc Z^* Z V_tc^* = G_tc G_tc^* (Eq. recomp_weight_full with P_tc isometric)."""
    rc = _rc(name)
    Z = rc.ZR if rows else rc.ZC
    for t, c, tc in _active(rc):
        G = explicit_Gtc(rc, t, c, rows)
        V = rc.dh2.full_basis(t, c)
        lhs = V @ Z[tc].conj().T @ Z[tc] @ V.conj().T
        rhs = G @ G.conj().T
        assert np.linalg.norm(lhs - rhs) <= 1e-10 * max(np.linalg.norm(rhs), 1e-300)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("rows", [True, False])
def test_singular_values_match_dense_algorithm(name, rows):
    """Section 3.1 on the explicit G_tc / G-hat_tc gives the singular values of Section 3.2."""
    rc = _rc(name)
    basis = rc.row if rows else rc.col
    for t, c, tc in _active(rc):
        ref = dense_singular_values(rc, t, c, rows)
        got = basis["sigma"][tc]
        nz = min(len(ref), len(got))
        scale = ref[0] if len(ref) else 1.0
        assert np.allclose(got[:nz], ref[:nz], rtol=0, atol=1e-9 * scale)
        assert np.all(ref[nz:] <= 1e-9 * scale) and np.all(got[nz:] <= 1e-9 * scale)


@pytest.mark.parametrize("name", CASES)
def test_new_bases_orthonormal_and_rank_rule(name):
    rc = _rc(name)
    for basis in (rc.row, rc.col):
        for t, c, tc in _active(rc):
            Q = basis["Q"][tc]
            k = basis["rank"][tc]
            assert Q.shape[1] == k
            assert np.allclose(Q.conj().T @ Q, np.eye(k), atol=1e-12)
            s = basis["sigma"][tc]
            tail = float((s[k:] ** 2).sum())
            assert tail <= rc.eps ** 2
            if k > 0:
                assert tail + s[k - 1] ** 2 > rc.eps ** 2   # k is the smallest such rank
            Qf = rc.full_new_basis(basis, t, c)
            assert np.allclose(Qf.conj().T @ Qf, np.eye(k), atol=1e-11)


def test_choose_rank_rules():
    s = np.array([1.0, 0.1, 1e-3, 1e-5, 1e-7])
    assert choose_rank(s, 1e-4, RANK_BLOCKREL) == 3
    assert choose_rank(s, 1e-2, RANK_BLOCKREL) == 2
    assert choose_rank(s, 1e-2, RANK_GLOBAL) == 2
    assert choose_rank(10 * s, 1e-4, RANK_GLOBAL) == 3
    assert choose_rank(np.zeros(0), 1e-4) == 0
    # spectral norm: the best rank-k error is sigma_{k+1}, so k = #{sigma_i > eps}
    assert choose_rank(s, 1e-4, RANK_SPECTRAL) == 3
    assert choose_rank(s, 1e-2, RANK_SPECTRAL) == 2
    assert choose_rank(s, 0.1, RANK_SPECTRAL) == 1      # sigma_2 = eps is allowed to go
    assert choose_rank(s, 2.0, RANK_SPECTRAL) == 0
    assert choose_rank(np.zeros(0), 1e-4, RANK_SPECTRAL) == 0


@pytest.mark.parametrize("name", ["dir320", "mixed1280"])
def test_spectral_rule_leaf_projection_error(name):
    """Spectral-norm error control: on every leaf pair the new basis Q leaves
    |G_tc - Q Q^* G_tc|_2 <= eps for the explicitly assembled weighted G_tc (numpy 2-norm,
    independent of the oracle's SVD path), and one column fewer would not; the ranks never
    exceed those of the Frobenius rule (sigma_{k+1} <= (sum_{i>k} sigma_i^2)^(1/2))."""
    rs = _rc(name, rule=RANK_SPECTRAL)
    rf = _rc(name)
    checked = 0
    for t, c, tc in _active(rs):
        assert rs.row["rank"][tc] <= rf.row["rank"][tc]
        assert rs.col["rank"][tc] <= rf.col["rank"][tc]
        if not rs.tree.is_leaf(t):
            continue
        G = explicit_Gtc(rs, t, c, True)
        if G.shape[1] == 0:
            continue
        Q = rs.row["Q"][tc]
        k = Q.shape[1]
        err = np.linalg.norm(G - Q @ (Q.conj().T @ G), 2)
        assert err <= rs.eps * (1 + 1e-8) + 1e-14
        if k > 0:
            Qm = Q[:, : k - 1]
            assert np.linalg.norm(G - Qm @ (Qm.conj().T @ G), 2) > rs.eps
        checked += 1
    assert checked > 0


@pytest.mark.parametrize("name", CASES)
def test_blockwise_error_bound(name):
    """|G_b - G~_b|_F <= eps sqrt(2 (p+1)) |G_b|_F for every admissible block (Section 3.1
    Pythagoras chain, applied to row and column bases)."""
    rc = _rc(name)
    d, tr = rc.dh2, rc.tree
    bound = rc.eps * math.sqrt(2 * (tr.depth + 1))
    worst = 0.0
    for b, (t, s, c) in enumerate(d.blocks.adm):
        Gb = d.full_basis(t, c) @ rc.S(b) @ d.full_basis(s, c).conj().T
        Gt = (rc.full_new_basis(rc.row, t, c) @ rc.Stilde[b]
              @ rc.full_new_basis(rc.col, s, c).conj().T)
        worst = max(worst, np.linalg.norm(Gb - Gt) / np.linalg.norm(Gb))
    assert worst <= bound


@pytest.mark.parametrize("name", CASES)
def test_matvec_equals_expanded_matrix(name):
    rc = _rc(name)
    A = rc.to_dense()
    x = synth.random_vector(rc.tree.n, 1809_0001)
    y = rc.matvec(x)
    assert np.linalg.norm(y - A @ x) <= 1e-13 * np.linalg.norm(A @ x)
    # and against the dense Galerkin matrix (reported accuracy of the whole method)
    G = rc.dh2.disc.dense(rc.dh2.kappa)
    assert np.linalg.norm(y - G @ x) <= 1e-2 * np.linalg.norm(G @ x)


def test_no_admissible_block_means_dense():
    """1280 triangles with the paper's parameters: every block is nearfield (DH^2 = G)."""
    rc = _rc("plain1280")
    assert len(rc.dh2.blocks.adm) == 0
    x = synth.random_vector(rc.tree.n, 1809_0001)
    G = rc.dh2.disc.dense(rc.dh2.kappa)
    assert np.linalg.norm(rc.matvec(x) - G @ x) <= 1e-13 * np.linalg.norm(G @ x)


def test_ancestor_sets():
    rc = _rc("dir320")
    tr = rc.tree
    for t, c, tc in list(_active(rc))[:50]:
        anc = ancestors(rc, t, c)
        assert anc[0] == (t, c)
        levels = [tr.level[a] for a, _ in anc]
        assert min(levels) >= 0 and max(levels) == tr.level[t]
