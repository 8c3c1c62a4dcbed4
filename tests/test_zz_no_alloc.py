"""The allocation-free matvec entry point against the ordinary one.

dh2_matvec_noalloc exists for callers that cannot call cudaMalloc when they need
the product (graph capture under another framework's allocator, real-time
loops, fixed memory budgets): it keeps its scratch in a fixed device array of
the library instead of per-matrix buffers.  Two calls in a row must both give
the product of dh2_matvec, within the tolerance of the other parity tests.
This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision, vec", [("mixed", "c64"), ("mixed", "c128"), ("fp64", "c128")])
def test_noalloc_matvec_matches_matvec_twice(precision, vec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_04384_gb300.build import build

    build()
    import paper_1809_04384_gb300 as dh2
    import synth
    from tests.cases import mesh, params
    from tests.gpu_common import TOL, rel

    v, f = mesh("mixed1280")
    p = params("mixed1280")
    tree = dh2.Tree(v, f, leaf_max=p["leaf"])
    prec = dh2.DH2_FP64 if precision == "fp64" else dh2.DH2_MIXED
    mat = dh2.Matrix(tree, p["kappa"], p["m"], p["eta2"], p["eps"], precision=prec, eta1=p["eta1"])
    dt = torch.complex128 if vec == "c128" else torch.complex64
    tol = TOL[precision]["matvec_same_ranks"]
    for seed in (11, 12):   # two calls in a row, different inputs
        x = torch.from_numpy(synth.random_vector(len(f), seed)).to(dt).cuda()
        y_ref = dh2.dh2_matvec(mat.handle, x, torch.empty_like(x))
        y = dh2.dh2_matvec_noalloc(mat.handle, x, torch.full_like(x, float("nan")))
        torch.cuda.synchronize()
        a = y.cpu().numpy().astype(np.complex128)
        b = y_ref.cpu().numpy().astype(np.complex128)
        assert np.all(np.isfinite(a))
        assert rel(a, b) <= tol

