"""Learned interpolation order and truncation rank (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

The paper fixes one interpolation order m for the whole matrix (Section 5:
"order m = 4 ... k = 4^3 = 64") and finds every rank k_tc by SVD truncation
at eps (Section 3.2).  The learned part predicts both per pair (t,c) from
geometry alone, before any interpolation is done, so that the analytic stage
(k = m^3) and the truncation buffers can be sized up front; the SVD
truncation still decides every rank.  The paper has no counterpart: every
definition below is this project's, written out plainly.

* ``features``: 8 numbers per pair (t, c), t on level l:
    f0 = kappa diam(B_t) / eta1                (oscillations across the box)
    f1 = theta_l / pi, theta_l = atan(sqrt(2) / m_l) the angular radius of a
         direction cone (a face square of width 2/m_l seen from the centre),
         theta_l = pi when D_l = {0}
    f2 = l / depth                              (0 when depth = 0)
    f3 >= f4 >= f5: the box extents hi - lo sorted, divided by diam(B_t)
    f6 = log2(#t) / 16
    f7 = max over admissible blocks b = (t, s, c) in row(t, c) of
         diam(B_t) / dist(B_t, B_s)  (0 without blocks or at dist = 0)
* ``probe_errors``: the interpolation error the method itself makes for a
  pair at order m (the label of the order): for the first 8 blocks of
  row(t, c), the first-kind Chebyshev interpolant of g_c(., y) on the padded
  box of t (the interpolation of Section 2, x side), compared with g_c at the
  3-point quadrature nodes of up to 8 elements of t (x) and of s (y);
  elements taken at positions offset + floor(j size / P), P = min(8, size).
  err(t, c, m) = max over blocks of max |g_c - interpolant| / max |g_c|.
* ``order_labels``: the smallest m in [3, 8] with err <= eps / 2 (the x and
  y sides of a block each contribute one such error), else 8.
* ``forward`` / ``loss_grad``: the MLP 8 -> 128 -> 128 -> 2 with ReLU hidden
  layers and a linear output, weights rounded to BF16 (round to nearest,
  ties to even) and biases kept in FP32, then evaluated in FP64; loss
  L = sum_{s,o} (y_so - t_so)^2 / (2 N).  Gradients are those of L with
  respect to the rounded weights (the FP32 master weights take them as
  theirs); ReLU'(z) = 1 iff z > 0.  Targets: t0 = m / 8, t1 = rank / 64.
* ``adam``: one Adam step (Kingma and Ba), bias-corrected moments.

Packed parameter order (FP32): W1 [128][8], b1 [128], W2 [128][128],
b2 [128], W3 [2][128], b3 [2]; 17922 values.

Pins (tests/test_oracle_learned.py): the gradient equals central finite
differences of the loss (brute force, FP64); BF16 rounding agrees with torch's
conversion and with hand-worked ties; the first Adam step has the closed form
p - lr g / (|g| + eps); the feature extents are unit vectors sorted
descending, the root pair's f0 is kappa diam / eta1 of the vertex box; the
probe error of a polynomial kernel of degree < m per axis vanishes to
rounding, and the probe error falls as m grows on a real block row.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import helmholtz_c

N_IN, N_HID, N_OUT = 8, 128, 2
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
ORDERS = tuple(range(3, 9))
M_SCALE, RANK_SCALE = 8.0, 64.0


def unpack(p):
    """Split the packed parameter vector into named arrays (views)."""
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name]).reshape(-1) for name, _ in SHAPES])


def bf16_round(w):
    """FP32 values rounded to the nearest BF16 (ties to even), returned as FP32."""
    u = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def effective(p32):
    """Parameters as the forward pass uses them: BF16 weights, FP32 biases, in FP64."""
    d = unpack(np.asarray(p32, dtype=np.float32))
    return {name: (bf16_round(v) if name.startswith("W") else v).astype(np.float64) for name, v in d.items()}


def forward_eff(e, X):
    """Pre-activations z1, z2, hidden h1, h2 and outputs y for inputs X (N x 8), given the
    effective FP64 parameters ``e`` (a dict as returned by ``effective``)."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ e["W1"].T + e["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ e["W2"].T + e["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ e["W3"].T + e["b3"]
    return z1, h1, z2, h2, y


def forward(p32, X):
    return forward_eff(effective(p32), X)


def loss_eff(e, X, T):
    y = forward_eff(e, X)[-1]
    return float(np.sum((y - np.asarray(T, dtype=np.float64)) ** 2) / (2.0 * len(X)))


def loss_grad_eff(e, X, T):
    """Loss and its gradient (packed layout) by the chain rule, layer by layer."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    z1, h1, z2, h2, y = forward_eff(e, X)
    n = len(X)
    dy = (y - T) / n
    g = {"W3": dy.T @ h2, "b3": dy.sum(axis=0)}
    dz2 = (dy @ e["W3"]) * (z2 > 0)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(axis=0)
    dz1 = (dz2 @ e["W2"]) * (z1 > 0)
    g["W1"], g["b1"] = dz1.T @ X, dz1.sum(axis=0)
    return float(np.sum((y - T) ** 2) / (2.0 * n)), pack(g)


def loss_grad(p32, X, T):
    return loss_grad_eff(effective(p32), X, T)


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns the new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed):
    """He-style uniform initial weights, zero biases (FP32)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            fan_in = shape[1]
            lim = math.sqrt(6.0 / fan_in)
            d[name] = rng.uniform(-lim, lim, size=shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d).astype(np.float32)


# --------------------------------------------------------------------------- features

def features(tree, dirs, blocks, pairs, kappa, eta1):
    """The 8 features of every pair (t, c), in pair order tc (array ntc x 8, FP64)."""
    diam = tree.diam()
    depth = tree.depth
    F = np.zeros((pairs.ntc, N_IN))
    for t in range(tree.nc):
        l = int(tree.level[t])
        ml = int(dirs.msplit[l])
        theta = math.atan(math.sqrt(2.0) / ml) if ml > 0 else math.pi
        ext = np.sort(tree.hi[t] - tree.lo[t])[::-1]
        dt = float(diam[t])
        for c in range(int(pairs.count[t])):
            tc = int(pairs.base[t] + c)
            f = F[tc]
            f[0] = kappa * dt / eta1
            f[1] = theta / math.pi
            f[2] = l / depth if depth > 0 else 0.0
            f[3:6] = ext / dt if dt > 0 else 0.0
            f[6] = math.log2(int(tree.size[t])) / 16.0
            close = 0.0
            for b in pairs.row[tc]:
                s = int(blocks.adm[b][1])
                g = np.maximum(np.maximum(tree.lo[t] - tree.hi[s], tree.lo[s] - tree.hi[t]), 0.0)
                dist = math.sqrt(float(g @ g))
                if dist > 0:
                    close = max(close, dt / dist)
            f[7] = close
    return F


# --------------------------------------------------------------------------- probe (labels)

PROBE_BLOCKS, PROBE_ELEMS = 8, 8


def sample_elements(tree, t):
    """Up to 8 elements of cluster t, at positions offset + floor(j size / P)."""
    size, off = int(tree.size[t]), int(tree.offset[t])
    P = min(PROBE_ELEMS, size)
    return np.array([tree.perm[off + (j * size) // P] for j in range(P)], dtype=np.int64)


def cheb_nodes(lo, hi, m):
    """First-kind Chebyshev nodes per axis on the box, half-widths padded to >= 1e-3 of the largest."""
    mid = (lo + hi) * 0.5
    half = (hi - lo) * 0.5
    half = np.maximum(half, 1e-3 * half.max())
    j = np.arange(m)
    ref = np.cos(math.pi * (2 * j + 1) / (2 * m))
    return mid[:, None] + half[:, None] * ref[None, :]       # (3, m)


def lagrange_1d(nodes, x):
    """l_j(x) for the nodes of one axis: (len(x), m), product form."""
    m = len(nodes)
    out = np.ones((len(x), m))
    for j in range(m):
        for i in range(m):
            if i != j:
                out[:, j] *= (x - nodes[i]) / (nodes[j] - nodes[i])
    return out


def tensor_nodes(nodes):
    """xi_nu for nu = nu_x + m nu_y + m^2 nu_z: (m^3, 3)."""
    m = nodes.shape[1]
    iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    return np.stack([nodes[0, ix.ravel()], nodes[1, iy.ravel()], nodes[2, iz.ravel()]], axis=1)


def tensor_lagrange(nodes, X):
    """L_nu(x) for x in X: (len(X), m^3), same index order as tensor_nodes."""
    lx, ly, lz = (lagrange_1d(nodes[a], X[:, a]) for a in range(3))
    return np.einsum("pk,pj,pi->pkji", lz, ly, lx).reshape(len(X), -1)


def probe_errors(disc, tree, dirs, blocks, pairs, kappa, kernel=None):
    """err[tc, m - 3] of the x-side interpolation for every pair and m in 3..8."""
    kernel = kernel or helmholtz_c
    err = np.zeros((pairs.ntc, len(ORDERS)))
    for tc in range(pairs.ntc):
        row = pairs.row[tc]
        if not row:
            continue
        t = int(np.searchsorted(pairs.base, tc, side="right") - 1)
        c = tc - int(pairs.base[t])
        cvec = dirs.dirs[int(tree.level[t])][c]
        X = disc.x3[sample_elements(tree, t)].reshape(-1, 3)
        for mi, m in enumerate(ORDERS):
            nodes = cheb_nodes(tree.lo[t], tree.hi[t], m)
            L = tensor_lagrange(nodes, X)
            xi = tensor_nodes(nodes)
            worst = 0.0
            for b in row[:PROBE_BLOCKS]:
                s = int(blocks.adm[b][1])
                Y = disc.x3[sample_elements(tree, s)].reshape(-1, 3)
                exact = kernel(X[:, None, :], Y[None, :, :], kappa, cvec)
                approx = L @ kernel(xi[:, None, :], Y[None, :, :], kappa, cvec)
                scale = np.abs(exact).max()
                worst = max(worst, float(np.abs(exact - approx).max() / scale))
            err[tc, mi] = worst
    return err


def order_labels(err, eps):
    """Smallest order m in [3, 8] whose probe error is at most eps / 2 (else 8)."""
    ok = err <= 0.5 * eps
    first = np.where(ok.any(axis=1), ok.argmax(axis=1), len(ORDERS) - 1)
    return np.asarray(ORDERS)[first]
