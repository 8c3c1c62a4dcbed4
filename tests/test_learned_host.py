"""Host logic of the learned-model training pipeline (no GPU): order labels, the label-threshold
calibration and the matrix-order rule, against brute force on hand-made data."""
import math

import numpy as np

from paper_1809_04384_gb300 import train_learned as TL


def _labels_brute(err, thresh):
    out = []
    for row in err:
        m = 8
        for mi, e in zip(range(3, 9), row):
            if e <= thresh:
                m = mi
                break
        out.append(m)
    return np.array(out)


def test_order_labels_brute_force():
    rng = np.random.default_rng(4)
    err = 10.0 ** rng.uniform(-9, -1, size=(500, 6))
    err = np.sort(err, axis=1)[:, ::-1]            # decreasing in m, as interpolation errors are
    err[::7] = rng.uniform(size=(len(err[::7]), 6))  # and some rows that never converge
    for thresh in (1e-6, 5e-5, 3.2e-3):
        np.testing.assert_array_equal(TL.order_labels(err, thresh), _labels_brute(err, thresh))


def test_calibrate_takes_the_largest_safe_threshold():
    eps = 1e-4
    # mesh A needs m = 6; its worst pair has errors 5e-3 at m = 5 and 1e-3 at m = 6
    errA = np.array([[1e-1, 1e-2, 5e-3, 1e-3, 1e-5, 1e-7], [1e-3, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9]])
    # mesh B needs m = 4: safe for every threshold of the grid
    errB = np.array([[1e-2, 1e-6, 1e-8, 1e-9, 1e-9, 1e-9]])
    data = [{"pairs": 2, "err": errA, "needed": 6}, {"pairs": 1, "err": errB, "needed": 4},
            {"pairs": 0}]
    c = TL.calibrate(data, eps)
    assert c == 32.0         # 32 eps = 3.2e-3: label 6; 64 eps = 6.4e-3 >= 5e-3: label 5, too low
    for cc in TL.C_GRID:
        safe = all(TL.order_labels(d["err"], cc * eps).max() >= d["needed"] for d in data if d["pairs"])
        assert safe == (cc <= c)


def test_rule_order_quantile_floor_clamp():
    # 100 pairs: the 99th percentile by nearest rank from below is the 99th smallest value
    p = np.linspace(3.0, 6.9, 100)
    want = int(math.floor(np.sort(p)[int(math.floor(0.99 * 99))]))
    assert TL.rule_order(p) == want == 6
    assert TL.rule_order(np.array([9.7])) == 8        # clamped above
    assert TL.rule_order(np.array([1.2, 2.0])) == 3   # clamped below
    # one outlier among many does not move the order (the maximum would)
    q = np.full(1000, 5.4)
    q[3] = 7.9
    assert TL.rule_order(q) == 5


def test_samples_targets():
    eps = 1e-4
    d = {"pairs": 2, "X": np.ones((2, 8), np.float32), "rank": np.array([12.0, 40.0]),
         "err": np.array([[1, 1, 1e-9, 1e-9, 1e-9, 1e-9], [1e-9] * 6])}
    X, T = TL.samples([d, {"pairs": 0}], 1.0, eps)
    np.testing.assert_allclose(T, [[5 / 8, 12 / 64], [3 / 8, 40 / 64]], rtol=1e-7)
    assert X.shape == (2, 8) and X.dtype == np.float32
