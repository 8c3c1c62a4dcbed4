"""GPU double-layer operator (dh2_options.layer = DH2_DOUBLE_LAYER) against the oracle.

The oracle is ``oracle/double_layer.py`` (pinned in tests/test_oracle_double_layer.py): the
kernel d/dn_y g, its dense Galerkin matrix, the interpolated DH^2 matrix with row basis V and
column basis W (normal derivative of the modified Lagrange polynomials), and the Section 3.2
recompression with separate basis weights R (from V) and R_W (from W).  Compared, as for the
single layer, on the invariants the paper fixes: the nearfield against the dense matrix, the
Gram matrices of R, R_W and of both total weights, the singular values and the product.
"""
import functools

import numpy as np
import pytest

from tests.gpu_common import TOL, form_kwargs, oracle_structure, rel, vec_dtype, x_vector

pytestmark = pytest.mark.gpu

CASES = ["dir320", "mixed1280", "lowfreq1280"]
PRECISIONS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_04384_gb300.build import build

    build()


@functools.lru_cache(maxsize=None)
def dlp_oracle(name):
    from oracle.double_layer import DoubleLayer, InterpolatedDLP, RecompressionDLP

    v, f, p, tr, dirs, bt = oracle_structure(name)
    layer = DoubleLayer(v, f)
    interp = InterpolatedDLP(layer, tr, dirs, bt, p["kappa"], p["m"])
    return layer, interp, RecompressionDLP(interp, p["eps"])


@functools.lru_cache(maxsize=None)
def dlp_gpu(name, precision):
    import paper_1809_04384_gb300 as dh2

    v, f, p, *_ = oracle_structure(name)
    tree = dh2.Tree(v, f, leaf_max=p["leaf"])
    mat = dh2.Matrix(tree, p["kappa"], p["m"], p["eta2"], p["eps"], eta1=p["eta1"], layer=dh2.DH2_DOUBLE_LAYER,
                     **form_kwargs(precision))
    return tree, mat


@pytest.mark.parametrize("precision", PRECISIONS)
def test_dlp_dense_case_equals_galerkin_matrix(precision):
    """1280 triangles with the paper's parameters: every block nearfield, so the product is the
    dense double-layer Galerkin matrix (zero diagonal)."""
    import torch

    layer, interp, rc = dlp_oracle("plain1280")
    _, mat = dlp_gpu("plain1280", precision)
    x = x_vector(rc.tree.n)
    K = layer.dense(interp.kappa)
    assert np.all(np.diag(K) == 0)
    y = mat.matvec(torch.from_numpy(x).to(vec_dtype(precision)).cuda()).cpu().numpy().astype(np.complex128)
    assert rel(y, K @ x) <= TOL[precision]["near"]


def _pair_tc(rc, tc):
    t = int(np.searchsorted(rc.pairs.base, tc, side="right") - 1)
    return t, int(tc - rc.pairs.base[t])


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", PRECISIONS)
def test_dlp_weights_and_singular_values(name, precision):
    import paper_1809_04384_gb300 as dh2

    _, interp, rc = dlp_oracle(name)
    _, mat = dlp_gpu(name, precision)
    assert mat.get_info().symmetric == 0
    tol = TOL[precision]
    for tc in np.nonzero(rc.pairs.active)[0]:
        t, c = _pair_tc(rc, tc)
        for which, Ro in ((dh2.DH2_X_R, rc.R[tc]), (dh2.DH2_X_RW, rc.RW[tc])):
            R = mat.pair(which, tc)
            assert R.shape == Ro.shape
            assert rel(R.conj().T @ R, Ro.conj().T @ Ro) <= tol["gram"], (which, tc)
        for which, Zo, leaf, P in ((dh2.DH2_X_ZROW, rc.ZR[tc], interp.leaf_basis, dh2.DH2_X_P),
                                   (dh2.DH2_X_ZCOL, rc.ZC[tc], interp.leaf_col_basis, dh2.DH2_X_PW)):
            Z = mat.pair(which, tc)
            if rc.tree.is_leaf(t):   # total weight in the coordinates of the leaf's orthonormal basis
                Pm = mat.pair(P, tc)
                B = leaf(t, c)
                lhs, rhs = Pm @ (Z.conj().T @ Z) @ Pm.conj().T, B @ (Zo.conj().T @ Zo) @ B.conj().T
            else:
                lhs, rhs = Z.conj().T @ Z, Zo.conj().T @ Zo
            if np.linalg.norm(rhs) == 0:
                assert np.linalg.norm(lhs) == 0
            else:
                assert rel(lhs, rhs) <= tol["gram"], (which, tc)
        for which, so in ((dh2.DH2_X_SROW, rc.row["sigma"][tc]), (dh2.DH2_X_SCOL, rc.col["sigma"][tc])):
            s = mat.pair(which, tc).real.ravel()
            n = min(len(s), len(so))
            if n:
                assert np.abs(s[:n] ** 2 - so[:n] ** 2).max() <= tol["sigma2"] * max(so[0], 1e-300) ** 2, (which, tc)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", PRECISIONS)
def test_dlp_matvec_matches_oracle(name, precision):
    import torch

    layer, interp, rc = dlp_oracle(name)
    _, mat = dlp_gpu(name, precision)
    x = x_vector(rc.tree.n)
    y_ref = rc.matvec(x)
    y = mat.matvec(torch.from_numpy(x).to(vec_dtype(precision)).cuda()).cpu().numpy().astype(np.complex128)
    rr, rcl = mat.ranks()
    act = np.nonzero(rc.pairs.active)[0]
    same = all(rr[tc] == rc.row["rank"][tc] and rcl[tc] == rc.col["rank"][tc] for tc in act)
    assert np.mean([rr[tc] != rc.row["rank"][tc] for tc in act]) <= 0.01
    assert rel(y, y_ref) <= (TOL[precision]["matvec_same_ranks"] if same else 2 * rc.eps)
    # both are equally close to the dense double-layer matrix
    Kx = layer.dense(interp.kappa) @ x
    assert rel(y, Kx) <= rel(y_ref, Kx) * 1.05 + 1e-6


@pytest.mark.parametrize("precision", PRECISIONS)
def test_dlp_direct_recompression_matches_oracle(precision):
    """The double layer through the direct recompression of the set-up (both bases evaluated
    and orthogonalised level by level) gives the oracle's product."""
    import torch

    import paper_1809_04384_gb300 as dh2

    _, _, rc = dlp_oracle("mixed1280")
    v, f, p, *_ = oracle_structure("mixed1280")
    tree = dh2.Tree(v, f, leaf_max=p["leaf"])
    mat = dh2.Matrix(tree, p["kappa"], p["m"], p["eta2"], p["eps"], eta1=p["eta1"], layer=dh2.DH2_DOUBLE_LAYER,
                     direct=1, **form_kwargs(precision))
    x = x_vector(rc.tree.n)
    y = mat.matvec(torch.from_numpy(x).to(vec_dtype(precision)).cuda()).cpu().numpy().astype(np.complex128)
    assert rel(y, rc.matvec(x)) <= max(TOL[precision]["matvec_same_ranks"], 2 * rc.eps if precision != "fp64" else 0)
