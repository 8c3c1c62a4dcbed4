"""Trains the learned order/rank model on labels that the method itself produces.

    python -m paper_1809_04384_gb300.train_learned [--meshes 40] [--steps 4000] [--out FILE]

Data (every step on the GPU through the library):

* meshes: ``synth.batch_meshes`` (spheres and ellipsoids of 1280-20480 triangles,
  semi-axes U[0.5, 2], kappa U[4, 16]; the configurations the model is meant for),
  leaf 32, eta1 10, eta2 1, eps 1e-4;
* features of every active pair (dh2_learned_features);
* order label: the smallest m in 3..8 whose x-side interpolation error
  (dh2_learned_probe) is at most eps / 2, since the two sides of a block each add
  one such error; 8 when none is;
* rank label: the row rank k_tc of a plain build at the reference order m_ref
  (dh2_export_ranks).

Targets are (m / 8, rank / 64); the loss is the mean squared error, minimised by
Adam (dh2_model_train_step) on shuffled mini-batches with a cosine learning-rate
decay.  The last meshes are held out for validation.  Prints one JSON line with the
data sizes, losses and validation statistics, and writes the FP32 parameters.
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


def order_labels(err, eps):
    """Smallest order with probe error <= eps / 2 per row of err (orders 3..8), else 8."""
    ok = err <= 0.5 * eps
    return np.where(ok.any(axis=1), ORDERS[ok.argmax(axis=1)], 8)


def mesh_samples(v, f, kappa, m_ref, eps=EPS):
    """(features [n, 8] float32, targets [n, 2] float32, order labels, ranks) of the active pairs."""
    tree = dh2.Tree(v, f, leaf_max=LEAF)
    F, active = dh2.learned_features(tree, kappa, ETA2, eta1=ETA1)
    err = dh2.learned_probe(tree, kappa, ETA2, eta1=ETA1)
    mat = dh2.Matrix(tree, kappa, m_ref, ETA2, eps, eta1=ETA1)
    rr, _ = mat.ranks()
    mat.close()
    tree.close()
    idx = np.nonzero(active)[0]
    lab = order_labels(err[idx], eps)
    rank = rr[idx].astype(np.float64)
    X = F.cpu().numpy()[idx]
    T = np.stack([lab / 8.0, rank / 64.0], axis=1).astype(np.float32)
    return X, T, lab, rank


def collect(count, seed, m_ref, log=print):
    data = []
    for i, (v, f, kappa) in enumerate(synth.batch_meshes(count, seed)):
        t0 = time.perf_counter()
        X, T, lab, rank = mesh_samples(v, f, kappa, m_ref)
        log(f"mesh {i}: {len(f)} triangles, kappa {kappa:.2f}: {len(X)} pairs, orders {np.bincount(lab, minlength=9)[3:]}"
            f", mean rank {rank.mean() if len(rank) else 0:.1f} ({time.perf_counter() - t0:.1f} s)")
        data.append((X, T))
    return data


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


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--meshes", type=int, default=40)
    ap.add_argument("--val", type=int, default=6, help="meshes held out for validation")
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
    data = collect(args.meshes, args.seed, args.m_ref, log=lambda s: print(s, file=sys.stderr))
    t_data = time.perf_counter() - t0
    tr, va = data[: args.meshes - args.val], data[args.meshes - args.val:]
    Xtr = np.concatenate([d[0] for d in tr]).astype(np.float32)
    Ttr = np.concatenate([d[1] for d in tr]).astype(np.float32)
    Xva = np.concatenate([d[0] for d in va]).astype(np.float32) if va else np.zeros((0, 8), np.float32)
    Tva = np.concatenate([d[1] for d in va]).astype(np.float32) if va else np.zeros((0, 2), np.float32)
    t1 = time.perf_counter()
    model, hist = train(Xtr, Ttr, args.steps, args.batch, args.lr, args.seed, args.seed + 1)
    t_train = time.perf_counter() - t1
    model.save(args.out)
    print(json.dumps({
        "samples_train": int(len(Xtr)), "samples_val": int(len(Xva)), "meshes": args.meshes, "m_ref": args.m_ref,
        "data_s": round(t_data, 2), "train_s": round(t_train, 2), "steps": args.steps, "batch": args.batch,
        "loss_first": hist[0][1], "loss_last": hist[-1][1],
        "train": evaluate(model, Xtr, Ttr), "val": evaluate(model, Xva, Tva), "out": args.out,
    }))


if __name__ == "__main__":
    main()
