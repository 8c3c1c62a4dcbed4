"""Pins of the learned-order oracle (oracle/learned.py) against brute force and closed forms."""
import math

import numpy as np
import pytest

from oracle import learned as L
from oracle.geometry import Discretisation
from oracle.structure import PairIndex
from tests.gpu_common import oracle_structure


def _rand_eff(seed):
    rng = np.random.default_rng(seed)
    e = {}
    for name, shape in L.SHAPES:
        e[name] = rng.normal(scale=0.3, size=shape)
    return e


def test_loss_gradient_matches_central_differences():
    """Chain-rule gradient of every parameter block against (L(p+h) - L(p-h)) / 2h in FP64."""
    rng = np.random.default_rng(1)
    e = _rand_eff(101)
    X = rng.normal(size=(6, L.N_IN))
    T = rng.normal(size=(6, L.N_OUT))
    z1, _, z2, _, _ = L.forward_eff(e, X)
    h = 1e-6
    # no pre-activation within reach of the step: the ReLU kink would spoil the difference
    assert min(np.abs(z1).min(), np.abs(z2).min()) > 1e3 * h
    _, g = L.loss_grad_eff(e, X, T)
    G = L.unpack(g)
    for name, shape in L.SHAPES:
        idx = [np.unravel_index(i, shape) for i in rng.choice(int(np.prod(shape)), size=min(40, int(np.prod(shape))), replace=False)]
        for ix in idx:
            ep = {k: v.copy() for k, v in e.items()}
            em = {k: v.copy() for k, v in e.items()}
            ep[name][ix] += h
            em[name][ix] -= h
            fd = (L.loss_eff(ep, X, T) - L.loss_eff(em, X, T)) / (2 * h)
            assert abs(fd - G[name][ix]) <= 1e-7 + 1e-6 * abs(fd), (name, ix, fd, G[name][ix])


def test_bf16_round_ties_and_library():
    one = np.float32(1.0)
    ulp = 2.0 ** -7                     # BF16 keeps 7 fraction bits
    cases = {
        1.0: 1.0,
        1.0 + ulp / 2: 1.0,             # tie, 1.0 has an even last bit
        1.0 + 1.5 * ulp: 1.0 + 2 * ulp, # tie, rounds up to the even neighbour
        1.0 + 0.75 * ulp: 1.0 + ulp,
        -(1.0 + 0.25 * ulp): -1.0,
    }
    for x, want in cases.items():
        assert float(L.bf16_round(np.float32(x))) == want, x
    assert one == L.bf16_round(one)
    torch = pytest.importorskip("torch")
    w = np.random.default_rng(1).normal(scale=3.0, size=4096).astype(np.float32)
    ref = torch.from_numpy(w).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(L.bf16_round(w), ref)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    p = rng.normal(size=100)
    g = rng.normal(size=100)
    lr, eps = 1e-3, 1e-8
    p1, m1, v1 = L.adam(p, g, np.zeros(100), np.zeros(100), 1, lr, eps=eps)
    np.testing.assert_allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)


def test_forward_uses_rounded_weights_and_fp32_biases():
    p = L.init_params(5)
    d = L.unpack(p.copy())
    d["b1"][:] = 0.1234567
    p = L.pack(d).astype(np.float32)
    e = L.effective(p)
    assert np.all(e["W2"] == L.bf16_round(L.unpack(p)["W2"]))
    assert np.all(e["b1"] == np.float32(0.1234567))


def _features_case(name):
    v, f, p, tr, dirs, bt = oracle_structure(name)
    pairs = PairIndex(tr, dirs, bt)
    F = L.features(tr, dirs, bt, pairs, p["kappa"], p["eta1"])
    return v, f, p, tr, dirs, bt, pairs, F


@pytest.mark.parametrize("name", ["mixed1280", "dir320"])
def test_feature_invariants(name):
    v, f, p, tr, dirs, bt, pairs, F = _features_case(name)
    ext = F[:, 3:6]
    np.testing.assert_allclose(np.sum(ext * ext, axis=1), 1.0, rtol=1e-13)
    assert np.all(ext[:, 0] >= ext[:, 1]) and np.all(ext[:, 1] >= ext[:, 2])
    diam = tr.diam()
    np.testing.assert_allclose(F[0, 0], p["kappa"] * diam[0] / p["eta1"], rtol=1e-15)
    for t in range(tr.nc):
        tcs = range(int(pairs.base[t]), int(pairs.base[t] + pairs.count[t]))
        l = int(tr.level[t])
        for tc in tcs:
            assert F[tc, 2] == l / tr.depth
            assert F[tc, 6] == math.log2(int(tr.size[t])) / 16.0
            if dirs.msplit[l] == 0:
                assert F[tc, 1] == 1.0
            else:
                assert 0.0 < F[tc, 1] < 0.5
            # admissible blocks satisfy (3b): diam_t <= eta2 dist
            assert (F[tc, 7] > 0) == bool(pairs.row[tc])
            assert F[tc, 7] <= p["eta2"] * (1 + 1e-12)


def test_probe_exact_for_polynomial_kernels():
    """A kernel that is a polynomial of degree <= 2 per axis in x is interpolated exactly for m >= 3."""
    v, f, p, tr, dirs, bt = oracle_structure("dir320")
    pairs = PairIndex(tr, dirs, bt)
    disc = Discretisation(v, f)

    def poly(x, y, kappa, c):
        return (x[..., 0] ** 2 * x[..., 1] - 3 * x[..., 2] ** 2 + x[..., 0] * x[..., 2] + 2.0) * (1.5 + y[..., 0]) + 0j

    err = L.probe_errors(disc, tr, dirs, bt, pairs, p["kappa"], kernel=poly)
    assert any(pairs.row[tc] for tc in range(pairs.ntc))
    assert err.max() < 1e-11


def test_probe_converges_and_labels():
    v, f, p, tr, dirs, bt = oracle_structure("mixed1280")
    pairs = PairIndex(tr, dirs, bt)
    disc = Discretisation(v, f)
    err = L.probe_errors(disc, tr, dirs, bt, pairs, p["kappa"])
    rows = [tc for tc in range(pairs.ntc) if pairs.row[tc]]
    med = np.median(err[rows], axis=0)
    assert np.all(np.diff(med) < 0), med
    lab = L.order_labels(err, 1e-4)
    assert lab.min() >= 3 and lab.max() <= 8
    # hand-made rows: first order under eps/2, none under (-> 8), already at m = 3
    e = np.array([[1, 1, 4e-5, 1e-6, 1e-7, 1e-8], [1] * 6, [0] * 6], dtype=float)
    np.testing.assert_array_equal(L.order_labels(e, 1e-4), [5, 8, 3])
