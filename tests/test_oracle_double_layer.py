"""Pins of the double-layer oracle (oracle/double_layer.py): derivative by finite differences,
Gauss's solid-angle identity, Green's representation formula, matrix invariants."""
import math

import numpy as np
import pytest

import synth
from oracle.double_layer import DoubleLayer, dlp_kernel, triangle_normals
from oracle.geometry import helmholtz


@pytest.mark.parametrize("kappa", [0.0, 3.0, 10.0])
def test_kernel_is_the_normal_derivative_of_g(kappa):
    rng = np.random.default_rng(11)
    x = rng.normal(size=(50, 3))
    y = rng.normal(size=(50, 3))
    n = rng.normal(size=(50, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    h = 1e-5
    fd = (helmholtz(x, y + h * n, kappa) - helmholtz(x, y - h * n, kappa)) / (2 * h)
    k = dlp_kernel(x, y, n, kappa)
    assert np.max(np.abs(fd - k) / np.abs(k)) < 1e-6


def test_icosphere_normals_point_outward():
    v, f = synth.icosphere(3)
    n = triangle_normals(v, f)
    cen = v[f].mean(axis=1)
    assert np.all(np.sum(n * cen, axis=1) > 0)
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, rtol=1e-14)


def test_gauss_identity_inside_and_outside():
    """kappa = 0: the potential of the constant density is -1 inside and 0 outside the closed
    surface, exactly for the polyhedron; the quadrature error falls under refinement."""
    inside = np.array([[0.0, 0.0, 0.0], [0.1, -0.2, 0.3]])
    outside = np.array([[0.0, 0.0, 3.0], [2.0, 1.0, 0.0]])
    errs = []
    for level in (2, 3, 4):
        v, f = synth.icosphere(level)
        D = DoubleLayer(v, f)
        p_in = D.potential(inside, 0.0)
        p_out = D.potential(outside, 0.0)
        assert np.all(np.abs(p_out) < 1e-6)
        errs.append(np.max(np.abs(p_in + 1.0)))
    assert errs[0] < 1e-4 and errs[1] < errs[0] / 8 and errs[2] < errs[1] / 8, errs


@pytest.mark.parametrize("kappa", [1.0, 3.0])
def test_green_representation_of_a_plane_wave(kappa):
    """u(x) = int [g du/dn - dg/dn_y u] for the plane wave u = exp(i kappa <d, y>) and x inside."""
    v, f = synth.icosphere(4)
    D = DoubleLayer(v, f)
    d = D.disc
    dirv = np.array([0.48, -0.6, 0.64])
    n = D.normals[:, None, :]
    u = np.exp(1j * kappa * (d.x3 @ dirv))
    du = 1j * kappa * (n @ dirv) * u
    for x in (np.array([0.1, -0.2, 0.3]), np.zeros(3)):
        s = np.sum(d.w3 * (helmholtz(x[None, None, :], d.x3, kappa) * du
                           - dlp_kernel(x[None, None, :], d.x3, n, kappa) * u))
        assert abs(s - np.exp(1j * kappa * (x @ dirv))) < 1e-6


def test_matrix_invariants():
    v, f = synth.icosphere(3)
    D = DoubleLayer(v, f)
    K0 = D.dense(0.0)
    assert np.all(np.diag(K0) == 0)
    assert np.abs(K0.imag).max() == 0.0
    # on the surface the identity gives -1/2: Galerkin row sums approach -|T_i| / 2
    ratio = K0.sum(axis=1).real / D.disc.area
    assert np.all(np.abs(ratio + 0.5) < 0.01)
    # entries of a sub-grid equal those of the full matrix
    K = D.dense(4.0)
    rows, cols = np.array([5, 77, 300]), np.array([0, 5, 1000, 1279])
    np.testing.assert_array_equal(D.entries(rows, cols, 4.0), K[np.ix_(rows, cols)])


def _dir320():
    from oracle.structure import build_block_tree, build_cluster_tree, build_directions
    from tests.cases import CASES

    level, kappa, leaf, eta1, eta2, m, eps = CASES["dir320"]
    v, f = synth.icosphere(level)
    tr = build_cluster_tree(v, f, leaf)
    dirs = build_directions(tr, kappa, eta1)
    bt = build_block_tree(tr, dirs, kappa, eta2)
    return v, f, tr, dirs, bt, kappa


def test_lagrange_gradients_reproduce_polynomial_gradients():
    from oracle.double_layer import InterpolatedDLP

    v, f, tr, dirs, bt, kappa = _dir320()
    I = InterpolatedDLP(DoubleLayer(v, f), tr, dirs, bt, kappa, 3)
    t = 5
    xi = I.cheb.points(t)
    p = lambda q: q[:, 0] ** 2 * q[:, 1] - 3 * q[:, 2] ** 2 + q[:, 0] * q[:, 2] + 2.0   # degree <= 2 per axis
    grad_p = lambda q: np.stack([2 * q[:, 0] * q[:, 1] + q[:, 2], q[:, 0] ** 2, -6 * q[:, 2] + q[:, 0]], axis=1)
    lo, hi = tr.lo[t], tr.hi[t]
    y = lo + (hi - lo) * np.random.default_rng(2).uniform(size=(40, 3))
    got = np.einsum("n,pna->pa", p(xi), I.lagrange_grad(t, y))
    np.testing.assert_allclose(got, grad_p(y), atol=1e-11 * np.abs(grad_p(y)).max())


def test_column_basis_is_the_normal_derivative_on_polynomials():
    """W applied to the nodal values of a polynomial p (degree <= m - 1 per axis) is the
    3-point rule of d/dn [exp(i kappa <y, c>) p(y)], here by central finite differences."""
    from oracle.double_layer import InterpolatedDLP

    v, f, tr, dirs, bt, kappa = _dir320()
    layer = DoubleLayer(v, f)
    I = InterpolatedDLP(layer, tr, dirs, bt, kappa, 3)
    p = lambda q: q[..., 0] ** 2 * q[..., 1] - 3 * q[..., 2] ** 2 + q[..., 0] * q[..., 2] + 2.0
    leaves = [t for t in range(tr.nc) if tr.is_leaf(t)]
    checked = 0
    for s in leaves[:6]:
        for c in range(dirs.count(int(tr.level[s]))):
            cvec = I.direction(s, c)
            W = I.leaf_col_basis(s, c)
            got = W @ p(I.cheb.points(s))
            idx = tr.indices(s)
            y = layer.disc.x3[idx]                                  # (#s, 3, 3)
            n = layer.normals[idx][:, None, :]
            h = 1e-6
            f_ = lambda q: np.exp(1j * kappa * (q @ cvec)) * p(q)
            dn = (f_(y + h * n) - f_(y - h * n)) / (2 * h)
            want = np.sum(layer.disc.w3[idx] * dn, axis=1)
            np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-9 * np.abs(want).max())
            checked += 1
    assert checked >= 6


def test_interpolated_dlp_product_and_convergence():
    from oracle.double_layer import InterpolatedDLP

    v, f, tr, dirs, bt, kappa = _dir320()
    layer = DoubleLayer(v, f)
    Kd = layer.dense(kappa)
    x = synth.random_vector(len(f), 5)
    errs = []
    for m in (3, 4, 5):
        I = InterpolatedDLP(layer, tr, dirs, bt, kappa, m)
        A = I.to_dense()
        assert np.linalg.norm(I.matvec(x) - A @ x) <= 1e-13 * np.linalg.norm(A @ x)
        errs.append(np.linalg.norm(A - Kd) / np.linalg.norm(Kd))
        # nearfield blocks are the dense entries themselves
        t, s = bt.near[0]
        np.testing.assert_array_equal(A[np.ix_(tr.indices(t), tr.indices(s))],
                                      Kd[np.ix_(tr.indices(t), tr.indices(s))])
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs


@pytest.fixture(scope="module")
def dlp_rc():
    from oracle.double_layer import InterpolatedDLP, RecompressionDLP

    v, f, tr, dirs, bt, kappa = _dir320()
    I = InterpolatedDLP(DoubleLayer(v, f), tr, dirs, bt, kappa, 3)
    return RecompressionDLP(I, 1e-4)


def test_dlp_basis_weights_gram(dlp_rc):
    """R_W^* R_W = W^* W and R^* R = V^* V with the bases expanded through Eq. (nested)."""
    rc = dlp_rc
    P = rc.pairs
    for l in range(rc.tree.depth + 1):
        for t, c in rc.active_pairs(l):
            tc = P.tc(t, c)
            for R, full in ((rc.R[tc], rc.dh2.full_basis), (rc.RW[tc], rc.dh2.full_col_basis)):
                B = full(t, c)
                g = B.conj().T @ B
                assert np.linalg.norm(R.conj().T @ R - g) <= 1e-11 * np.linalg.norm(g)


def test_dlp_recompression_bound_orthonormality_product(dlp_rc):
    rc = dlp_rc
    d, tr = rc.dh2, rc.tree
    # new bases orthonormal
    for basis in (rc.row, rc.col):
        for l in range(tr.depth + 1):
            for t, c in rc.active_pairs(l):
                Q = rc.full_new_basis(basis, t, c)
                if Q.shape[1]:
                    assert np.linalg.norm(Q.conj().T @ Q - np.eye(Q.shape[1])) < 1e-12
    # blockwise error bound of the Pythagoras chain
    bound = rc.eps * math.sqrt(2 * (tr.depth + 1))
    for b, (t, s, c) in enumerate(d.blocks.adm):
        Gb = d.full_basis(t, c) @ rc.S(b) @ d.full_col_basis(s, c).conj().T
        Gt = rc.full_new_basis(rc.row, t, c) @ rc.Stilde[b] @ rc.full_new_basis(rc.col, s, c).conj().T
        assert np.linalg.norm(Gb - Gt) <= bound * np.linalg.norm(Gb)
    # the product equals the expanded recompressed matrix
    A = rc.to_dense()
    x = synth.random_vector(tr.n, 1809_0001)
    assert np.linalg.norm(rc.matvec(x) - A @ x) <= 1e-13 * np.linalg.norm(A @ x)
    # W != V: row and column ranks are not all equal
    rows = [rc.row["rank"][tc] for tc in rc.row["rank"]]
    cols = [rc.col["rank"][tc] for tc in rc.col["rank"]]
    assert rows != cols


def _case(name):
    from oracle.structure import build_block_tree, build_cluster_tree, build_directions
    from tests.cases import CASES

    level, kappa, leaf, eta1, eta2, m, eps = CASES[name]
    v, f = synth.icosphere(level)
    tr = build_cluster_tree(v, f, leaf)
    dirs = build_directions(tr, kappa, eta1)
    bt = build_block_tree(tr, dirs, kappa, eta2)
    return v, f, tr, dirs, bt, kappa, m


def test_no_admissible_block_gives_the_dense_matrix():
    from oracle.double_layer import InterpolatedDLP

    v, f, tr, dirs, bt, kappa, m = _case("plain1280")
    assert len(bt.adm) == 0
    layer = DoubleLayer(v, f)
    I = InterpolatedDLP(layer, tr, dirs, bt, kappa, m)
    np.testing.assert_array_equal(I.to_dense(), layer.dense(kappa))


def test_nested_column_basis_is_exact_without_oscillation():
    """kappa = 0 (c = 0): the transfers reproduce the father's polynomials exactly, so the
    column basis built through them equals the father's directly integrated normal
    derivatives (leaf_col_basis applied to the father's own elements and nodes)."""
    from oracle.double_layer import InterpolatedDLP

    v, f, tr, dirs, bt, kappa, m = _case("laplace1280")
    I = InterpolatedDLP(DoubleLayer(v, f), tr, dirs, bt, kappa, m)
    checked = 0
    for t in range(tr.nc):
        if tr.is_leaf(t) or tr.level[t] < tr.depth - 2:
            continue
        nested = I.full_col_basis(t, 0)
        direct = I.leaf_col_basis(t, 0)
        assert np.linalg.norm(nested - direct) <= 1e-11 * np.linalg.norm(direct)
        checked += 1
    assert checked > 0
