"""GPU reference rows of the Galerkin matrix (dh2_dense_rows) against the oracle's dense rows."""
import numpy as np
import pytest

import synth
from oracle.geometry import Discretisation
from tests.gpu_common import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("level,kappa", [(3, 4.0), (3, 0.0), (4, 16.0)])
def test_dense_rows_match_oracle(level, kappa):
    import torch

    import paper_1809_04384_gb300 as dh2
    from paper_1809_04384_gb300.build import build

    build()
    v, f = synth.ellipsoid(level, (1.0, 0.7, 1.3))
    x = synth.random_vector(len(f), 1809_0007)
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(len(f), size=40, replace=False))
    rows[0] = 0
    rows[-1] = len(f) - 1          # first and last element
    tree = dh2.Tree(v, f)
    got = dh2.dh2_dense_rows(tree.handle, kappa, rows, torch.from_numpy(x).cuda())
    want = Discretisation(v, f).dense_rows_matvec(rows, x, kappa)
    assert rel(got, want) <= 1e-12, rel(got, want)
    # no rows: nothing to do
    assert dh2.dh2_dense_rows(tree.handle, kappa, [], torch.from_numpy(x).cuda()).shape == (0,)
    with pytest.raises(dh2.DH2Error):
        dh2.dh2_dense_rows(tree.handle, kappa, [len(f)], torch.from_numpy(x).cuda())
