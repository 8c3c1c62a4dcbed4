"""Batched builds and products (dh2_build_dh2_batch, dh2_matvec_batch).

Concurrent builds on several streams must give the matrices of one-at-a-time
builds: the same ranks and the same products (the kernels and their inputs are
the same; only the interleaving on the GPU differs).  One mesh of the batch is
also checked against the oracle's recompressed matvec, as the single-build
parity tests do.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _meshes():
    import synth

    from tests.cases import mesh, params

    p = params("mixed1280")
    v0, f0 = mesh("mixed1280")
    v1, f1 = synth.ellipsoid(2, np.array([1.5, 0.7, 1.1]))
    v2, f2 = synth.icosphere(2)
    v3, f3 = synth.ellipsoid(3, np.array([0.6, 1.3, 0.9]))
    return p, [(v0, f0, p["kappa"]), (v1, f1, 5.0), (v2, f2, 3.0), (v3, f3, 6.5)]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_build_matches_single_builds_and_oracle(precision):
    import torch

    import paper_1809_04384_gb300 as dh2
    import synth
    from tests.gpu_common import TOL, oracle_recompression, rel, x_vector

    p, meshes = _meshes()
    prec = dh2.DH2_FP64 if precision == "fp64" else dh2.DH2_MIXED
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    tol = TOL[precision]
    trees = [dh2.Tree(v, f, leaf_max=p["leaf"]) for v, f, _ in meshes]
    kappas = [k for _, _, k in meshes]
    mats = dh2.build_batch(trees, kappas, p["m"], p["eta2"], p["eps"], precision=prec, eta1=p["eta1"],
                           nstreams=3)
    singles = [dh2.Matrix(t, k, p["m"], p["eta2"], p["eps"], precision=prec, eta1=p["eta1"])
               for t, k in zip(trees, kappas)]
    xs = [torch.from_numpy(synth.random_vector(len(f), 40 + i)).to(dt).cuda() for i, (_, f, _) in enumerate(meshes)]
    ys = dh2.matvec_batch(mats, xs)
    torch.cuda.synchronize()
    for i, (mb, ms) in enumerate(zip(mats, singles)):
        rb, cb = mb.ranks()
        rs, cs = ms.ranks()
        assert np.array_equal(rb, rs) and np.array_equal(cb, cs), f"mesh {i}: ranks differ"
        y_single = ms.matvec(xs[i]).cpu().numpy().astype(np.complex128)
        y_batch = ys[i].cpu().numpy().astype(np.complex128)
        assert np.all(np.isfinite(y_batch))
        assert rel(y_batch, y_single) <= tol["matvec_same_ranks"], f"mesh {i}"
    # mesh 0 is the mixed1280 parity case: same product as the oracle's recompression
    rc = oracle_recompression("mixed1280")
    x = x_vector(rc.tree.n)
    y0 = mats[0].matvec(torch.from_numpy(x).to(dt).cuda()).cpu().numpy().astype(np.complex128)
    assert rel(y0, rc.matvec(x)) <= max(tol["matvec_same_ranks"], 2 * rc.eps if precision == "mixed" else 0)
    for m in mats + singles:
        m.close()


def test_batch_rejects_point_mode_tree_and_clears_outputs():
    import paper_1809_04384_gb300 as dh2
    import synth

    v, f = synth.icosphere(1)
    good = dh2.Tree(v, f, leaf_max=8)
    points = dh2.Tree(v, None, leaf_max=8)
    with pytest.raises(dh2.DH2Error) as e:
        dh2.build_batch([good, points], [1.0, 1.0], 3, 1.0, 1e-4)
    assert e.value.status == dh2.DH2_EINVAL


def test_matvec_batch_rejects_repeated_matrix():
    import torch

    import paper_1809_04384_gb300 as dh2
    import synth

    v, f = synth.icosphere(2)
    tree = dh2.Tree(v, f, leaf_max=8)
    mat = dh2.Matrix(tree, 3.0, 3, 4.0, 1e-4, eta1=1.0)
    x = torch.from_numpy(synth.random_vector(len(f), 3)).to(torch.complex64).cuda()
    with pytest.raises(dh2.DH2Error) as e:
        dh2.matvec_batch([mat, mat], [x, x.clone()])
    assert e.value.status == dh2.DH2_EINVAL
