"""Shared fixtures for the GPU parity tests: oracle results cached per case."""
import functools

import numpy as np

import synth
from oracle.geometry import Discretisation
from oracle.interp import InterpolatedDH2
from oracle.recompress import Recompression
from oracle.structure import build_block_tree, build_cluster_tree, build_directions
from tests.cases import mesh, params

# Floating-point tolerances per precision, relative.  gram: Frobenius error of R^*R and
# Z^*Z; sigma2: |s_gpu^2 - s_oracle^2| / s_1^2 (the truncation forms the Gram matrix of
# V Z^* in FP64, so squared singular values carry an absolute error ~ u s_1^2); matvec:
# relative 2-norm error against the oracle's recompressed matvec when all ranks agree.
# The mixed form computes products and weight QRs in complex FP32 (u = 6e-8) with
# error growth over the stacked rows.
TOL = {
    "fp64": dict(gram=1e-10, sigma2=1e-12, matvec_same_ranks=1e-9, near=1e-12, rank_slack=1e-6),
    "mixed": dict(gram=1e-4, sigma2=1e-4, matvec_same_ranks=1e-5, near=1e-5, rank_slack=2e-2),
}


@functools.lru_cache(maxsize=None)
def oracle_structure(name):
    v, f = mesh(name)
    p = params(name)
    tr = build_cluster_tree(v, f, p["leaf"])
    dirs = build_directions(tr, p["kappa"], p["eta1"])
    bt = build_block_tree(tr, dirs, p["kappa"], p["eta2"])
    return v, f, p, tr, dirs, bt


@functools.lru_cache(maxsize=None)
def oracle_recompression(name):
    v, f, p, tr, dirs, bt = oracle_structure(name)
    d = InterpolatedDH2(Discretisation(v, f), tr, dirs, bt, p["kappa"], p["m"])
    return Recompression(d, p["eps"])


@functools.lru_cache(maxsize=None)
def gpu_matrix(name, precision):
    import paper_1809_04384_gb300 as dh2

    v, f, p, *_ = oracle_structure(name)
    tree = dh2.Tree(v, f, leaf_max=p["leaf"])
    prec = dh2.DH2_FP64 if precision == "fp64" else dh2.DH2_MIXED
    mat = dh2.Matrix(tree, p["kappa"], p["m"], p["eta2"], p["eps"], precision=prec, eta1=p["eta1"])
    return tree, mat


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def x_vector(n):
    return synth.random_vector(n, 1809_0001)


def check_total_weight(mat, rc, tc, which, Zo, tol):
    """Z^*Z of the GPU total weight against the oracle's, on the invariant the paper fixes.

    Leaf pairs keep their total weight in the coordinates of the orthonormal basis P of
    V_tc = P R_tc, so P Z'^* Z' P^* is compared with V Z^* Z V^*; other pairs compare
    Z^* Z directly (k x k).
    """
    import paper_1809_04384_gb300 as dh2

    P_ = rc.pairs
    t = int(np.searchsorted(P_.base, tc, side="right") - 1)
    c = int(tc - P_.base[t])
    Z = mat.pair(which, tc)
    if rc.tree.is_leaf(t):
        Pm = mat.pair(dh2.DH2_X_P, tc)
        V = rc.dh2.leaf_basis(t, c)
        lhs = Pm @ (Z.conj().T @ Z) @ Pm.conj().T
        rhs = V @ (Zo.conj().T @ Zo) @ V.conj().T
    else:
        assert Z.shape == Zo.shape
        lhs, rhs = Z.conj().T @ Z, Zo.conj().T @ Zo
    if np.linalg.norm(rhs) == 0:
        assert np.linalg.norm(lhs) == 0
        return
    assert rel(lhs, rhs) <= tol, (which, tc, rel(lhs, rhs))
