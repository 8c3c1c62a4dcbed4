"""Trains the learned order/rank model on labels that the method itself produces.

    python -m paper_1809_04384_gb300.train_learned [--meshes 40] [--steps 4000] [--out FILE]

Data (every step on the GPU through the library):

* meshes: ``synth.batch_meshes`` (spheres and ellipsoids of 1280-20480 triangles,
  semi-axes U[0.5, 2], kappa U[4, 16]; the configurations the model is meant for) and
  ``synth.directional_meshes`` (20480 triangles, kappa U[28, 40], whose admissible blocks
  reach directional levels, as those of larger meshes at higher kappa do), leaf 32, eta1 10,
  eta2 1, eps 1e-4;
* features of every active pair (dh2_learned_features);
* the x-side interpolation error of every pair at m = 3..8 (dh2_learned_probe);
* the order each mesh needs: the smallest m in 4..7 whose built matrix has a
  relative product error <= eps on sampled rows against the FP64 Galerkin rows
  (dh2_dense_rows), 8 if none has;
* order label of a pair: the smallest m whose probe error is <= c eps, 8 if none
  is.  The threshold c is calibrated on the training meshes: the largest c from a
  grid for which the largest label of every mesh still reaches the order the mesh
  needs (the build takes the largest predicted order, so a smaller c only costs
  time);
* rank label: the row rank k_tc of the plain build at the reference order m_ref
  (dh2_export_ranks).

The build takes the 99th percentile of the orders predicted for a matrix's pairs,
rounded down.  After training, the order unit's bias is raised by the smallest
offset (grid of 0.05) for which that rule reaches the needed order on every
training mesh.

Targets are (m / 8, rank / 64); the loss is the mean squared error, minimised by
Adam (dh2_model_train_step) on shuffled mini-batches with a cosine learning-rate
decay.  The last meshes are held out for validation.  Prints one JSON line with the
data sizes, the calibration, losses and validation statistics, and writes the FP32
parameters.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

import paper_1809_04384_gb300 as dh2  # noqa: E402

TRAIN_SEED = 18090040
ETA1, ETA2, EPS, LEAF = 10.0, 1.0, 1e-4, 32
ORDERS = np.arange(3, 9)


C_GRID = (0.5, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 128.0)
GLOBAL_ORDERS = (4, 5, 6, 7)


def order_labels(err, thresh):
    """Smallest order with probe error <= thresh per row of err (orders 3..8), else 8."""
    ok = err <= thresh
    return np.where(ok.any(axis=1), ORDERS[ok.argmax(axis=1)], 8)


def product_error(mat, tree, kappa, x, rows):
    import torch

    y = mat.matvec(torch.from_numpy(x).to(torch.complex64).cuda()).cpu().numpy().astype(np.complex128)
    ref = dh2.dh2_dense_rows(tree.handle, kappa, rows, torch.from_numpy(x).cuda())
    return float(np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref))


def mesh_data(v, f, kappa, m_ref, eps=EPS, nrows=64, seed=0):
    """Features, probe errors and ranks of the active pairs, and the order the mesh needs."""
    tree = dh2.Tree(v, f, leaf_max=LEAF)
    F, active = dh2.learned_features(tree, kappa, ETA2, eta1=ETA1)
    idx = np.nonzero(active)[0]
    out = {"X": F.cpu().numpy()[idx], "pairs": len(idx)}
    if len(idx) == 0:
        tree.close()
        return out
    out["err"] = dh2.learned_probe(tree, kappa, ETA2, eta1=ETA1)[idx]
    x = synth.random_vector(len(f), seed)
    rows = np.sort(np.random.default_rng(seed + 1).choice(len(f), size=min(nrows, len(f)), replace=False))
    gerr = {}
    for m in sorted(set(GLOBAL_ORDERS) | {m_ref}):
        mat = dh2.Matrix(tree, kappa, m, ETA2, eps, eta1=ETA1)
        if m == m_ref:
            out["rank"] = mat.ranks()[0][idx].astype(np.float64)
        if m in GLOBAL_ORDERS:
            gerr[m] = product_error(mat, tree, kappa, x, rows)
        mat.close()
    tree.close()
    out["global_err"] = gerr
    out["needed"] = next((m for m in GLOBAL_ORDERS if gerr[m] <= eps), 8)
    return out


def collect(count, seed, m_ref, log=print, directional=0):
    data = []
    meshes = synth.batch_meshes(count, seed) + synth.directional_meshes(directional, seed + 7)
    for i, (v, f, kappa) in enumerate(meshes):
        t0 = time.perf_counter()
        d = mesh_data(v, f, kappa, m_ref, seed=seed + 100 + i)
        if d["pairs"]:
            log(f"mesh {i}: {len(f)} triangles, kappa {kappa:.2f}: {d['pairs']} pairs, needs m = {d['needed']} "
                f"(errors {', '.join(f'{m}: {e:.2e}' for m, e in d['global_err'].items())}), "
                f"mean rank {d['rank'].mean():.1f} ({time.perf_counter() - t0:.1f} s)")
        data.append(d)
    return data


def calibrate(data, eps):
    """Largest c of the grid for which every mesh's largest label reaches the order it needs."""
    best = C_GRID[0]
    for c in C_GRID:
        if all(order_labels(d["err"], c * eps).max() >= d["needed"] for d in data if d["pairs"]):
            best = c
    return best


def samples(data, c, eps):
    X = [d["X"] for d in data if d["pairs"]]
    T = [np.stack([order_labels(d["err"], c * eps) / 8.0, d["rank"] / 64.0], axis=1) for d in data if d["pairs"]]
    if not X:
        return np.zeros((0, 8), np.float32), np.zeros((0, 2), np.float32)
    return np.concatenate(X).astype(np.float32), np.concatenate(T).astype(np.float32)


def train(Xtr, Ttr, steps, batch, lr, seed, init_seed):
    """Adam on the GPU; returns the model and the loss history (every 100 steps)."""
    import torch

    rng = np.random.default_rng(init_seed)
    params = []
    for shape in [(128, 8), (128,), (128, 128), (128,), (2, 128), (2,)]:
        if len(shape) == 2:
            lim = math.sqrt(6.0 / shape[1])
            params.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            params.append(np.zeros(shape))
    model = dh2.Model(np.concatenate(params).astype(np.float32))
    X = torch.from_numpy(Xtr).cuda()
    T = torch.from_numpy(Ttr).cuda()
    n = len(X)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    perm = torch.randperm(n, device="cuda", generator=g)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    pos = 0
    for step in range(steps):
        if pos + batch > n:
            perm = torch.randperm(n, device="cuda", generator=g)
            pos = 0
        sel = perm[pos:pos + batch]
        pos += batch
        cur = lr * 0.5 * (1.0 + math.cos(math.pi * step / steps)) + 1e-5
        model.train_step(X[sel].contiguous(), T[sel].contiguous(), cur, loss)
        if step % 100 == 0 or step == steps - 1:
            hist.append((step, float(loss.item())))
    return model, hist


def evaluate(model, X, T):
    import torch

    if len(X) == 0:
        return {}
    Y = model.forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    m_hat = np.clip(np.rint(Y[:, 0] * 8.0), 3, 8)
    m_lab = np.rint(T[:, 0] * 8.0)
    r_hat = np.maximum(Y[:, 1] * 64.0, 0.0)
    r_lab = T[:, 1].astype(np.float64) * 64.0
    cap = np.ceil(1.25 * r_hat) + 4
    return {
        "mse": float(np.mean((Y - T) ** 2) / 2.0),
        "order_exact": float(np.mean(m_hat == m_lab)),
        "order_under": float(np.mean(m_hat < m_lab)),
        "order_max_pred": int(m_hat.max()), "order_max_label": int(m_lab.max()),
        "rank_mae": float(np.mean(np.abs(r_hat - r_lab))),
        "cap_exceeded": float(np.mean(r_lab > cap)),
    }


ORDER_QUANTILE = 0.99


def rule_order(pred_m):
    """The order a learned build takes from the predicted orders of its pairs."""
    q = np.sort(pred_m)[int(math.floor(ORDER_QUANTILE * (len(pred_m) - 1)))]
    return int(math.floor(min(8.0, max(3.0, q))))


def predicted_orders(model, data):
    import torch

    return [model.forward(torch.from_numpy(d["X"].astype(np.float32)).cuda()).cpu().numpy()[:, 0].astype(np.float64)
            * 8.0 for d in data if d["pairs"]]


def calibrate_offset(model, data):
    """Smallest offset (grid 0.05, at most 3) for which the rule reaches every mesh's needed order."""
    preds = predicted_orders(model, data)
    needed = [d["needed"] for d in data if d["pairs"]]
    for k in range(61):
        delta = 0.05 * k
        if all(rule_order(p + delta) >= n for p, n in zip(preds, needed)):
            return delta
    return 3.0


def mesh_orders(model, data):
    """(order the learned build takes, order the mesh needs) per mesh with pairs."""
    needed = [d["needed"] for d in data if d["pairs"]]
    return [(rule_order(p), n) for p, n in zip(predicted_orders(model, data), needed)]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--meshes", type=int, default=40)
    ap.add_argument("--val", type=int, default=6, help="meshes held out for validation")
    ap.add_argument("--directional", type=int, default=8, help="directional meshes added to the training meshes")
    ap.add_argument("--seed", type=int, default=TRAIN_SEED)
    ap.add_argument("--m-ref", type=int, default=6)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=dh2.LEARNED_WEIGHTS)
    args = ap.parse_args(argv)
    from paper_1809_04384_gb300.build import build

    build()
    t0 = time.perf_counter()
    data = collect(args.meshes, args.seed, args.m_ref, log=lambda s: print(s, file=sys.stderr),
                   directional=args.directional)
    t_data = time.perf_counter() - t0
    # validation: the last args.val meshes of the sphere/ellipsoid family; every directional
    # mesh trains
    tr = data[: args.meshes - args.val] + data[args.meshes:]
    va = data[args.meshes - args.val: args.meshes]
    c = calibrate(tr, EPS)
    Xtr, Ttr = samples(tr, c, EPS)
    Xva, Tva = samples(va, c, EPS)
    t1 = time.perf_counter()
    model, hist = train(Xtr, Ttr, args.steps, args.batch, args.lr, args.seed, args.seed + 1)
    t_train = time.perf_counter() - t1
    stats_tr, stats_va = evaluate(model, Xtr, Ttr), evaluate(model, Xva, Tva)
    delta = calibrate_offset(model, tr)
    params = model.params()
    params[-2] += np.float32(delta / 8.0)       # b3[0], the order unit's bias
    model = dh2.Model(params)
    model.save(args.out)
    print(json.dumps({
        "samples_train": int(len(Xtr)), "samples_val": int(len(Xva)), "meshes": args.meshes,
        "directional_meshes": args.directional, "m_ref": args.m_ref,
        "label_threshold_eps": c, "order_offset": delta, "data_s": round(t_data, 2), "train_s": round(t_train, 2), "steps": args.steps,
        "batch": args.batch, "loss_first": hist[0][1], "loss_last": hist[-1][1],
        "train": stats_tr, "val": stats_va,
        "orders_train": mesh_orders(model, tr), "orders_val": mesh_orders(model, va), "out": args.out,
    }))


if __name__ == "__main__":
    main()
