"""Failure reporting of a build, injected on the host (no GPU fault is ever caused).

dh2_options.fault makes the host find the device error bit that a tensor-core wait that
gave up (DH2_FAULT_TIMEOUT) or a non-finite value (DH2_FAULT_NONFINITE) would have set
after the projection stage, or makes the build's first device allocation fail
(DH2_FAULT_ALLOC).  The build must return the documented status (DH2_ETIMEOUT,
DH2_ENUMERIC, DH2_ENOMEM), hand out no matrix, and leave the library usable.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_04384_gb300.build import build

    build()
    import paper_1809_04384_gb300 as dh2
    from tests.cases import mesh, params

    v, f = mesh("dir320")
    p = params("dir320")
    return dh2, dh2.Tree(v, f, leaf_max=p["leaf"]), p


@pytest.mark.parametrize("fault, status", [(1, -4), (2, -5), (3, -2)])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_injected_fault_returns_status(case, fault, status, precision):
    import torch

    dh2, tree, p = case
    prec = dh2.DH2_FP64 if precision == "fp64" else dh2.DH2_MIXED
    assert (dh2.DH2_FAULT_TIMEOUT, dh2.DH2_FAULT_NONFINITE, dh2.DH2_FAULT_ALLOC) == (1, 2, 3)
    assert (dh2.DH2_ETIMEOUT, dh2.DH2_ENUMERIC, dh2.DH2_ENOMEM) == (-4, -5, -2)
    with pytest.raises(dh2.DH2Error) as ei:
        dh2.Matrix(tree, p["kappa"], p["m"], p["eta2"], p["eps"], precision=prec, eta1=p["eta1"], fault=fault)
    assert ei.value.status == status
    if fault == 1:
        assert "not usable" in str(ei.value)
    # the library (and the next build on this thread) is unaffected
    mat = dh2.Matrix(tree, p["kappa"], p["m"], p["eta2"], p["eps"], precision=prec, eta1=p["eta1"])
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    x = torch.ones(mat.n, dtype=dt, device="cuda")
    y = mat.matvec(x).cpu().numpy()
    assert np.all(np.isfinite(y))


def test_bad_fault_hook_is_rejected(case):
    dh2, tree, p = case
    with pytest.raises(dh2.DH2Error) as ei:
        dh2.Matrix(tree, p["kappa"], p["m"], p["eta2"], p["eps"], eta1=p["eta1"], fault=7)
    assert ei.value.status == dh2.DH2_EINVAL
