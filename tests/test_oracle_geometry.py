"""Pins of the oracle's kernel, quadrature and dense Galerkin matrix (Eq. 1, Eq. 2)."""
import math

import numpy as np
import pytest

import synth
from oracle.geometry import (BARY3, BARY7, W3, W7, Discretisation, helmholtz,
                             helmholtz_c, quad_points, triangle_areas)


def _ref_triangle_integral(a, b):
    """int over the unit reference triangle of x^a y^b = a! b! / (a+b+2)!  (closed form)."""
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("bary,w,degree", [(BARY3, W3, 2), (BARY7, W7, 5)])
def test_rules_exact_on_monomials(bary, w, degree):
    v = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    tri = np.array([[0, 1, 2]])
    x = quad_points(v, tri, bary)[0]
    area = triangle_areas(v, tri)[0]
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            q = area * np.sum(w * x[:, 0] ** a * x[:, 1] ** b)
            assert q == pytest.approx(_ref_triangle_integral(a, b), rel=1e-13, abs=1e-15)
    # one degree more is not integrated exactly (the pin can fail)
    errs = [abs(area * np.sum(w * x[:, 0] ** a * x[:, 1] ** (degree + 1 - a))
                - _ref_triangle_integral(a, degree + 1 - a)) for a in range(degree + 2)]
    assert max(errs) > 1e-6


def test_weights_sum_to_area():
    v, f = synth.icosphere(2)
    d = Discretisation(v, f)
    assert np.allclose(d.w3.sum(1), d.area, rtol=1e-14)
    assert np.allclose(d.w7.sum(1), d.area, rtol=1e-14)
    # a triangle's area from the cross product equals Heron's formula
    p = v[f[0]]
    a, b, c = (np.linalg.norm(p[1] - p[0]), np.linalg.norm(p[2] - p[1]), np.linalg.norm(p[0] - p[2]))
    s = 0.5 * (a + b + c)
    assert d.area[0] == pytest.approx(math.sqrt(s * (s - a) * (s - b) * (s - c)), rel=1e-10)


def test_kernel_closed_forms():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((50, 3))
    y = rng.standard_normal((50, 3))
    r = np.linalg.norm(x - y, axis=1)
    # kappa = 0: Laplace kernel 1/(4 pi r)
    assert np.allclose(helmholtz(x, y, 0.0), 1.0 / (4 * math.pi * r), rtol=1e-15)
    # |g| = 1/(4 pi r) and the phase is kappa r
    g = helmholtz(x, y, 3.0)
    assert np.allclose(np.abs(g), 1.0 / (4 * math.pi * r), rtol=1e-14)
    assert np.allclose(np.angle(g * np.exp(-3j * r)), 0.0, atol=1e-13)
    # plane-wave split: g = exp(i kappa <x-y,c>) g_c; g_0 = g
    c = np.array([0.3, -0.4, math.sqrt(1 - 0.25)])
    gc = helmholtz_c(x, y, 3.0, c)
    assert np.allclose(np.exp(3j * ((x - y) @ c)) * gc, g, rtol=1e-13)
    assert np.allclose(helmholtz_c(x, y, 3.0, np.zeros(3)), g, rtol=1e-15)
    # symmetry g(x,y) = g(y,x)
    assert np.allclose(helmholtz(y, x, 3.0), g, rtol=1e-15)


def test_dense_symmetric_and_laplace_real():
    v, f = synth.icosphere(2)
    d = Discretisation(v, f)
    G = d.dense(5.0)
    off = ~np.eye(d.n, dtype=bool)
    assert np.allclose(G[off], G.T[off], rtol=1e-13)
    G0 = d.dense(0.0)
    assert np.all(G0.imag == 0.0)
    assert np.all(G0.real > 0.0)
    assert np.all(np.diag(G0).real > G0.real.max(axis=1) * 0.999)   # the self-interaction dominates


def test_entry_against_independent_tensor_rule():
    """A far pair: the 3x3 rule agrees with an independent 7x7 tensor rule."""
    v, f = synth.icosphere(3)
    d = Discretisation(v, f)
    i, j = 0, 700
    ci = v[f[i]].mean(0)
    cj = v[f[j]].mean(0)
    assert np.linalg.norm(ci - cj) > 0.5
    ref = 0.0 + 0.0j
    for p in range(7):
        for q in range(7):
            xp = sum(BARY7[p, a] * v[f[i, a]] for a in range(3))
            yq = sum(BARY7[q, a] * v[f[j, a]] for a in range(3))
            r = np.linalg.norm(xp - yq)
            ref += W7[p] * W7[q] * d.area[i] * d.area[j] * np.exp(2j * r) / (4 * math.pi * r)
    got = d.entries(np.array([i]), np.array([j]), 2.0)[0, 0]
    assert abs(got - ref) / abs(ref) < 1e-5


def test_sampled_rows_match_dense():
    v, f = synth.icosphere(2)
    d = Discretisation(v, f)
    x = synth.random_vector(d.n, 3)
    rows = np.array([0, 17, 200, 319])
    assert np.allclose(d.dense_rows_matvec(rows, x, 4.0), (d.dense(4.0) @ x)[rows], rtol=1e-13)
