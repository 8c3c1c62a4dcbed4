"""GPU parity of the learned order/rank model: the MLP forward, gradient and Adam kernels, the
features and the interpolation-error probe against the oracle (oracle/learned.py), and the
learned build (order choice, rank caps and their fallback) against the plain build."""
import numpy as np
import pytest

from oracle import learned as OL
from oracle.geometry import Discretisation
from oracle.structure import PairIndex
from tests.gpu_common import gpu_matrix, oracle_structure, rel, x_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dh2():
    import paper_1809_04384_gb300 as pkg
    from paper_1809_04384_gb300.build import build

    build()
    return pkg


def _params(seed):
    p = OL.init_params(seed)
    d = OL.unpack(p.astype(np.float64))
    rng = np.random.default_rng(seed + 1)
    for name in ("b1", "b2", "b3"):
        d[name][:] = rng.normal(scale=0.1, size=d[name].shape)
    return OL.pack(d).astype(np.float32)


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.5, size=(n, OL.N_IN)).astype(np.float32)
    T = rng.uniform(0.3, 1.0, size=(n, OL.N_OUT)).astype(np.float32)
    return X, T


def _blocks(v):
    out, o = {}, 0
    for name, shape in OL.SHAPES:
        k = int(np.prod(shape))
        out[name] = v[o:o + k]
        o += k
    return out


@pytest.mark.parametrize("n", [1, 37, 1000, 9733])
def test_mlp_forward_matches_oracle(dh2, n):
    import torch

    p = _params(11)
    X, _ = _inputs(n, 5)
    model = dh2.Model(p)
    Y = model.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    Yo = OL.forward(p, X)[-1]
    assert rel(Y, Yo) <= 1e-5, rel(Y, Yo)


@pytest.mark.parametrize("n", [37, 1000, 9733])
def test_mlp_gradient_matches_oracle(dh2, n):
    """Ragged tiles (n not a multiple of 32) and several tiles per CTA (n > 152 x 32)."""
    import torch

    p = _params(12)
    X, T = _inputs(n, 6)
    model = dh2.Model(p)
    g, L = model.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    Lo, go = OL.loss_grad(p, X, T)
    assert abs(float(L.item()) - Lo) <= 1e-5 * Lo
    gb, gob = _blocks(g.cpu().numpy().astype(np.float64)), _blocks(go)
    for name, _ in OL.SHAPES:
        assert rel(gb[name], gob[name]) <= 1e-4, (name, rel(gb[name], gob[name]))


def test_adam_step_matches_oracle(dh2):
    import torch

    p = _params(13)
    X, T = _inputs(500, 7)
    model = dh2.Model(p)
    lr = 1e-3
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    model.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), lr, loss)
    p1 = model.params().astype(np.float64)
    Lo, go = OL.loss_grad(p, X, T)
    po, _, _ = OL.adam(p.astype(np.float64), go, np.zeros_like(go), np.zeros_like(go), 1, lr)
    assert abs(float(loss.item()) - Lo) <= 1e-5 * Lo
    big = np.abs(go) > 1e-6          # a gradient at rounding level may flip sign: step bounded by lr
    assert np.max(np.abs(p1 - po)[big]) <= 1e-6
    assert np.max(np.abs(p1 - po)) <= 1.01 * lr
    # the BF16 copies follow: a forward pass uses the stepped weights
    Y = model.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    assert rel(Y, OL.forward(p1.astype(np.float32), X)[-1]) <= 1e-5


def test_training_reduces_loss(dh2):
    import torch

    p = _params(14)
    rng = np.random.default_rng(8)
    X = rng.uniform(0, 1, size=(4096, 8)).astype(np.float32)
    T = np.stack([0.5 + 0.3 * X[:, 0] * X[:, 1], 0.2 + 0.5 * X[:, 7]], axis=1).astype(np.float32)
    model = dh2.Model(p)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    L0 = float(model.grad(Xd, Td)[1].item())
    for _ in range(300):
        model.train_step(Xd, Td, 2e-3)
    L1 = float(model.grad(Xd, Td)[1].item())
    assert L1 < 0.05 * L0, (L0, L1)


@pytest.mark.parametrize("name", ["mixed1280", "dir320", "dir1280"])
def test_features_match_oracle(dh2, name):
    v, f, p, tr, dirs, bt = oracle_structure(name)
    pairs = PairIndex(tr, dirs, bt)
    Fo = OL.features(tr, dirs, bt, pairs, p["kappa"], p["eta1"])
    tree = dh2.Tree(v, f, leaf_max=p["leaf"])
    F, active = dh2.learned_features(tree, p["kappa"], p["eta2"], eta1=p["eta1"])
    F = F.cpu().numpy().astype(np.float64)
    assert F.shape == Fo.shape
    np.testing.assert_array_equal(active, pairs.active)
    np.testing.assert_allclose(F, Fo.astype(np.float32), rtol=2e-7, atol=1e-7)


@pytest.mark.parametrize("name", ["dir320", "mixed1280"])
def test_probe_matches_oracle(dh2, name):
    v, f, p, tr, dirs, bt = oracle_structure(name)
    pairs = PairIndex(tr, dirs, bt)
    erro = OL.probe_errors(Discretisation(v, f), tr, dirs, bt, pairs, p["kappa"])
    tree = dh2.Tree(v, f, leaf_max=p["leaf"])
    err = dh2.learned_probe(tree, p["kappa"], p["eta2"], eta1=p["eta1"])
    assert err.shape == erro.shape
    # both FP64; the interpolant sums up to 512 terms, so rounding leaves ~1e-12 of |g_c|
    np.testing.assert_allclose(err, erro, rtol=1e-6, atol=1e-11)
    # the order labels agree wherever no error sits within rounding of eps / 2
    eps = p["eps"]
    clear = np.all(np.abs(erro - 0.5 * eps) > 1e-6 * eps, axis=1)
    np.testing.assert_array_equal(OL.order_labels(err, eps)[clear], OL.order_labels(erro, eps)[clear])


def _const_model(dh2, m, rank):
    """A model whose output is the constant (m / 8, rank / 64) (all weights zero)."""
    p = np.zeros(OL.NPARAMS, dtype=np.float32)
    p[-2] = m / 8.0
    p[-1] = rank / 64.0
    return dh2.Model(p)


@pytest.mark.parametrize("name", ["lowfreq1280", "mixed1280"])
def test_learned_build_rank_caps_and_fallback(dh2, name):
    """Caps below the ranks redo the truncation with the structural bounds; caps above them
    shrink the truncation buffers.  Either way ranks and product equal the plain build's.
    (The caps apply to the pairs of levels with D_l = {0}; both cases have such pairs of
    rank above 4.)"""
    import torch

    v, f, p, *_ = oracle_structure(name)
    tree, plain = gpu_matrix(name, "mixed")
    rr0, rc0 = plain.ranks()
    x = torch.from_numpy(x_vector(plain.n)).to(torch.complex64).cuda()
    y0 = plain.matvec(x).cpu().numpy()
    b0 = plain.info.truncation_bytes
    maxr = int(max(rr0.max(), rc0.max()))
    assert maxr > 4
    # caps of 4 columns (estimate 0) are exceeded in both passes (in the row pass only where
    # the column pass is its mirror); caps of exactly the largest rank (estimate
    # (maxr - 4) / 1.25) never are
    passes = 1 if plain.get_info().symmetric else 2
    for cap_rank, retries in ((0.0, passes), ((maxr - 4) / 1.25, 0)):
        model = _const_model(dh2, p["m"], cap_rank)
        mat = dh2.Matrix(tree, p["kappa"], 1, p["eta2"], p["eps"], eta1=p["eta1"], model=model)
        info = mat.get_info()
        assert info.learned_m == p["m"] and info.m == p["m"]
        assert info.rank_cap_retries == retries
        rr, rc = mat.ranks()
        np.testing.assert_array_equal(rr, rr0)
        np.testing.assert_array_equal(rc, rc0)
        y = mat.matvec(x).cpu().numpy()
        assert rel(y, y0) <= 1e-6
        if retries == 0:
            assert info.truncation_bytes <= b0
        else:
            assert info.truncation_bytes == b0


def test_learned_build_takes_predicted_order(dh2):
    v, f, p, *_ = oracle_structure("dir320")
    tree = dh2.Tree(v, f, leaf_max=p["leaf"])
    for m in (3, 4, 6):
        mat = dh2.Matrix(tree, p["kappa"], 5, p["eta2"], p["eps"], eta1=p["eta1"], model=_const_model(dh2, m, 64))
        assert mat.info.m == m and mat.info.k == m ** 3 and mat.info.learned_m == m
    # out-of-range predictions are clamped to [3, 8]
    mat = dh2.Matrix(tree, p["kappa"], 5, p["eta2"], p["eps"], eta1=p["eta1"], model=_const_model(dh2, 11, 64))
    assert mat.info.m == 8


def test_trained_model_gain(dh2):
    """What the shipped model gains over the plain method on a mesh outside its training set
    (an ellipsoid of 20480 triangles, kappa 12): the plain method at the configured order
    m = 5 misses eps = 1e-4 on sampled rows; the learned build chooses an order that meets
    it, and its truncated bases take less memory than a plain build at that order."""
    import torch

    import synth

    v, f = synth.ellipsoid(5, (1.3, 0.8, 1.0))
    kappa, eps = 12.0, 1e-4
    tree = dh2.Tree(v, f)
    x = synth.random_vector(len(f), 1809_0001)
    rows = np.sort(np.random.default_rng(1809_0002).choice(len(f), size=256, replace=False))
    ref = dh2.dh2_dense_rows(tree.handle, kappa, rows, torch.from_numpy(x).cuda())
    xd = torch.from_numpy(x).to(torch.complex64).cuda()

    def err(mat):
        return rel(mat.matvec(xd).cpu().numpy()[rows], ref)

    plain5 = dh2.Matrix(tree, kappa, 5, 1.0, eps)
    learned = dh2.Matrix(tree, kappa, 5, 1.0, eps, model=dh2.Model.load())
    m = learned.info.m
    plain_m = dh2.Matrix(tree, kappa, m, 1.0, eps)
    assert err(plain5) > eps
    assert m > 5 and err(learned) <= eps
    assert abs(err(learned) - err(plain_m)) <= 1e-3 * err(plain_m)
    np.testing.assert_array_equal(learned.ranks()[0], plain_m.ranks()[0])
    assert learned.info.truncation_bytes < plain_m.info.truncation_bytes


def test_learned_build_on_a_directional_mesh(dh2):
    """A mesh outside the training set whose admissible blocks reach directional levels (the
    20480-triangle sphere at kappa 36): the learned build caps only the pairs of levels with
    D_l = {0}, so no rank exceeds its cap (no truncation pass is redone), its truncated bases
    take less memory than a plain build at the same order, its ranks are the plain ones and
    its product meets eps on sampled rows."""
    import torch

    import synth

    v, f = synth.icosphere(5)
    kappa, eps = 36.0, 1e-4
    tree = dh2.Tree(v, f)
    learned = dh2.Matrix(tree, kappa, 5, 1.0, eps, model=dh2.Model.load())
    m = learned.info.m
    plain_m = dh2.Matrix(tree, kappa, m, 1.0, eps)
    # the structure has directional pairs
    adm, _, active = learned.blocks()
    assert any(learned.directions(l)[0] > 0 for l in range(learned.info.depth + 1))
    assert learned.info.rank_cap_retries == 0
    assert learned.info.truncation_bytes < plain_m.info.truncation_bytes
    np.testing.assert_array_equal(learned.ranks()[0], plain_m.ranks()[0])
    x = synth.random_vector(len(f), 1809_0001)
    rows = np.sort(np.random.default_rng(1809_0002).choice(len(f), size=128, replace=False))
    ref = dh2.dh2_dense_rows(tree.handle, kappa, rows, torch.from_numpy(x).cuda())
    y = learned.matvec(torch.from_numpy(x).to(torch.complex64).cuda()).cpu().numpy()[rows]
    assert rel(y, ref) <= eps


def test_learned_caps_leave_directional_pairs_alone(dh2):
    """On a block tree whose pairs of rank above 4 all lie on directional levels (dir1280),
    caps of 4 columns are never exceeded: directional pairs keep the structural bound."""
    import torch

    v, f, p, *_ = oracle_structure("dir1280")
    tree, plain = gpu_matrix("dir1280", "mixed")
    mat = dh2.Matrix(tree, p["kappa"], 1, p["eta2"], p["eps"], eta1=p["eta1"], model=_const_model(dh2, p["m"], 0.0))
    assert mat.get_info().rank_cap_retries == 0
    np.testing.assert_array_equal(mat.ranks()[0], plain.ranks()[0])
    x = torch.from_numpy(x_vector(plain.n)).to(torch.complex64).cuda()
    assert rel(mat.matvec(x).cpu().numpy(), plain.matvec(x).cpu().numpy()) <= 1e-6
