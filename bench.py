#!/usr/bin/env python
"""Benchmark of the GB300 hybrid DH^2 build + matvec.

One step = the whole hot path on one synthetic workload: cluster tree,
directions, block tree, nearfield, directional interpolation, basis weights,
total weights (rows and columns), SVD truncation, projection (dh2_build_tree +
dh2_build_dh2), then one DH^2 matvec (dh2_matvec).

Workload (default): unit sphere, icosahedral refinement to 20480 flat
triangles, kappa = 16 (kappa h ~ 0.5), leaf <= 32, eta1 = 10, eta2 = 1,
Chebyshev m = 5 (k = 125), eps = 1e-4, seeded N(0,1) + i N(0,1) vectors.

Prints ONE JSON line (rank 0).  `value` = build seconds per step (device time
with CUDA events on the launching stream); the matvec throughput (algorithmic
GB/s: every stored coefficient + the vectors, once) and its error against
sampled dense Galerkin rows are reported beside it, together with the plain
FP64 GPU form of the same build, and the learned order/rank model on the same
workload (the order it chooses, its build time and error, and the truncation memory
against a plain build at that order).  `--learned` makes the timed builds themselves
choose their order with the shipped model.  Before the timed region the library's
autotuner (dh2_autotune) picks the weight-QR tile shapes on the workload itself; every
build of the run uses them (`--no-autotune`: library defaults; `--qr-tpc a,b,c`: fixed).  The error reference is the FP64 Galerkin
rows, evaluated on the GPU by the library (dh2_dense_rows).  `--impl reference`
times the CPU oracle (the reference arm) on a bounded sample of the same workload.

    python bench.py [--steps K] [--warmup W] [--precision mixed|fp64] [--impl ours|reference] [--learned]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (mesh, kappa, leaf, eta1, eta2, m, eps); mesh ("icosphere", L) has 20 * 4^L
    # triangles, ("cube", q) is the surface of [-1/2, 1/2]^3 with 12 q^2 triangles
    "sphere20480": (("icosphere", 5), 16.0, 32, 10.0, 1.0, 5, 1e-4),
    "sphere1280": (("icosphere", 3), 4.0, 32, 10.0, 1.0, 4, 1e-4),
    "sphere5120": (("icosphere", 4), 8.0, 32, 10.0, 1.0, 5, 1e-4),     # same kappa h, for profiling captures
    "sphere81920": (("icosphere", 6), 32.0, 32, 10.0, 1.0, 5, 1e-4),
    "sphere327680": (("icosphere", 7), 64.0, 64, 10.0, 1.0, 5, 1e-4),
    "cube196608": (("cube", 128), 48.0, 64, 10.0, 1.0, 5, 1e-4),
}


def workload_mesh(name):
    import synth

    kind, size = WORKLOADS[name][0]
    return synth.icosphere(size) if kind == "icosphere" else synth.cube(size)
METRIC = "DH2 build s + matvec GB/s at rel.err≤1e-4 vs dense; vs plain FP64 GPU form"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="sphere20480", choices=list(WORKLOADS))
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU form")
    ap.add_argument("--error-rows", type=int, default=256)
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-mesh batched build")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the host-buffer end-to-end builds (a second matrix may not fit beside the first)")
    ap.add_argument("--batch-meshes", type=int, default=64)
    ap.add_argument("--learned", action="store_true",
                    help="the timed builds choose the order with the shipped learned model")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-order comparison")
    ap.add_argument("--m", type=int, default=0, help="override the workload's interpolation order")
    ap.add_argument("--no-autotune", action="store_true", help="library default tile shapes, no autotuning")
    ap.add_argument("--qr-tpc", default="", help="fixed weight-QR threads per column 'a,b,c' (skips autotuning)")
    ap.add_argument("--qr-group-rows", type=int, default=0, help="fixed weight-QR row-group size (with --qr-tpc)")
    return ap.parse_args()


def workload_config(name):
    (kind, size), kappa, leaf, eta1, eta2, m, eps = WORKLOADS[name]
    if kind == "icosphere":
        ntri, mesh = 20 * 4 ** size, "unit sphere, icosahedral refinement"
    else:
        ntri, mesh = 12 * size ** 2, f"surface of the cube [-1/2,1/2]^3, {size} x {size} squares per face"
    return dict(workload=f"{kind}{ntri}", mesh=mesh, triangles=ntri, kappa=kappa, leaf=leaf, eta1=eta1,
                eta2=eta2, m=m, k=m ** 3, eps=eps)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for name, val in zip(names, s[4:8]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ----------------------------------------------------------------------------- CPU oracle baseline

def oracle_sample_seconds(name, out_queue=None):
    """Times the oracle on a bounded sample of the workload (runs in a child process).

    Sample: the full structure phase (cluster tree, directions, block tree) of the
    workload, plus the complete build (nearfield + interpolation + recompression) of
    the mesh patch under one level-3 cluster (~1/8 of the triangles, same mesh
    density, kappa, leaf, m, eps).  The patch costs are scaled to the full workload by
    its admissible-block and nearfield-entry counts.
    """
    import synth
    from oracle.geometry import Discretisation
    from oracle.interp import InterpolatedDH2
    from oracle.recompress import Recompression
    from oracle.structure import build_block_tree, build_cluster_tree, build_directions

    _, kappa, leaf, eta1, eta2, m, eps = WORKLOADS[name]
    v, f = workload_mesh(name)
    t0 = time.perf_counter()
    tr = build_cluster_tree(v, f, leaf)
    dirs = build_directions(tr, kappa, eta1)
    bt = build_block_tree(tr, dirs, kappa, eta2)
    t_struct = time.perf_counter() - t0
    near_full = int(sum(tr.size[t] * tr.size[s] for t, s in bt.near))
    nadm_full = len(bt.adm)
    plevel = min(3, tr.depth)
    t = tr.level_start[plevel]
    idx = np.sort(tr.indices(t))
    used, inv = np.unique(f[idx], return_inverse=True)
    vs, fs = v[used], inv.reshape(-1, 3).astype(np.int32)
    t0 = time.perf_counter()
    tr2 = build_cluster_tree(vs, fs, leaf)
    d2 = build_directions(tr2, kappa, eta1)
    b2 = build_block_tree(tr2, d2, kappa, eta2)
    dh = InterpolatedDH2(Discretisation(vs, fs), tr2, d2, b2, kappa, m)
    t1 = time.perf_counter()
    rc = Recompression(dh, eps)
    t2 = time.perf_counter()
    for (a, b) in b2.near:
        dh.nearfield_block(a, b)
    t3 = time.perf_counter()
    near_s = int(sum(tr2.size[a] * tr2.size[b] for a, b in b2.near))
    t_recomp = t2 - t1
    t_near = t3 - t2
    est = t_struct + t_recomp * nadm_full / max(len(b2.adm), 1) + t_near * near_full / max(near_s, 1)
    res = dict(value=est, sample_seconds=t_struct + (t3 - t0), patch_triangles=len(fs),
               patch_adm=len(b2.adm), patch_near_entries=near_s, full_adm=nadm_full, full_near_entries=near_full,
               t_struct=t_struct, t_recomp=t_recomp, t_near=t_near)
    return res


def run_oracle_child(name):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample_seconds(%r)))" % (ROOT, name))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_obj(res):
    return {"value": res["value"], "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle structure phase on the full mesh + full oracle build of a "
                       f"{res['patch_triangles']}-triangle patch (one level-3 cluster) of the same sphere; "
                       f"recompression scaled by admissible blocks ({res['patch_adm']} -> {res['full_adm']}), "
                       f"nearfield by entries ({res['patch_near_entries']} -> {res['full_near_entries']}); "
                       f"{res['sample_seconds']:.1f} s of single-threaded CPU work")}


# ----------------------------------------------------------------------------- GPU arm

TILES = {}   # weight-QR tile shapes chosen by the autotuner for this run (empty: library defaults)


def gpu_build(pkg, v, f, cfg, precision, stream, model=None):
    tree = pkg.Tree(v, f, leaf_max=cfg["leaf"], stream=stream)
    mat = pkg.Matrix(tree, cfg["kappa"], cfg["m"], cfg["eta2"], cfg["eps"], precision=precision,
                     eta1=cfg["eta1"], model=model, stream=stream, **TILES)
    tree.close()
    return mat


def autotune(pkg, v, f, cfg, precision, stream):
    """dh2_autotune on the workload itself (outside the timed region): sets TILES and returns
    the report for the JSON line."""
    import time as _t

    tree = pkg.Tree(v, f, leaf_max=cfg["leaf"], stream=stream)
    base = pkg.options(eta1=cfg["eta1"], precision=precision)
    t0 = _t.perf_counter()
    tuned, t_ms, b_ms = pkg.dh2_autotune(tree.handle, cfg["kappa"], cfg["m"], cfg["eta2"], cfg["eps"], base, reps=2,
                                         stream=stream)
    wall = _t.perf_counter() - t0
    tree.close()
    TILES.update(qr_tpc=tuple(int(t) for t in tuned.qr_tpc), qr_group_rows=int(tuned.qr_group_rows))
    return {"qr_threads_per_column": list(TILES["qr_tpc"]), "qr_group_rows": TILES["qr_group_rows"],
            "qr_ms_per_build_tuned": t_ms, "qr_ms_per_build_default": b_ms, "tuning_s": wall,
            "note": "0 = library default (8, 4, 2 threads per column; 1024-row groups)"}


def time_steps(pkg, torch, v, f, cfg, precision, x_dev, steps, warmup, stream, model=None):
    """Device-timed steps: build (tree + DH^2) and one matvec, CUDA events on `stream`."""
    build_ms, mv_ms = [], []
    mats = []
    for i in range(warmup + steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        y = torch.empty_like(x_dev)
        torch.cuda.synchronize()
        e0.record(stream)
        mat = gpu_build(pkg, v, f, cfg, precision, stream, model)
        e1.record(stream)
        mat.matvec(x_dev, y, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            build_ms.append(e0.elapsed_time(e1))
            mv_ms.append(e1.elapsed_time(e2))
            mats.append(mat)
        else:
            mat.close()
    return build_ms, mv_ms, mats


def matvec_repeat_ms(torch, mat, x_dev, reps, stream):
    y = torch.empty_like(x_dev)
    for _ in range(3):
        mat.matvec(x_dev, y, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        mat.matvec(x_dev, y, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def sampled_dense_error(pkg, torch, mat, tree, kappa, x, rows_count, seed):
    """Relative 2-norm error of the product on sampled rows against the FP64 Galerkin rows,
    which the library evaluates on the GPU (dh2_dense_rows, every column by quadrature)."""
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(mat.n, size=min(rows_count, mat.n), replace=False))
    dt = torch.complex64 if mat.precision == 1 else torch.complex128
    y = mat.matvec(torch.from_numpy(x).to(dt).cuda()).cpu().numpy().astype(np.complex128)
    ref = pkg.dh2_dense_rows(tree.handle, kappa, rows, torch.from_numpy(x).to(torch.complex128).cuda())
    return float(np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref))


def learned_measure(pkg, torch, v, f, cfg, x, ref_tree, rows_count, err_configured, stream, with_fp64=True):
    """The learned order/rank model on the workload: the order it chooses, the build time
    (CUDA events, tree included, after one warm-up build), the sampled error against the
    FP64 Galerkin rows, and the truncation memory against a plain build at the same order;
    next to the error of the configured order."""
    model = pkg.Model.load()
    x_dev = torch.from_numpy(x).to(torch.complex64).cuda()
    ms, mats = time_steps(pkg, torch, v, f, cfg, pkg.DH2_MIXED, x_dev, 2, 1, stream, model)[0::2]
    mat = mats[-1]
    info = mat.get_info()
    err = sampled_dense_error(pkg, torch, mat, ref_tree, cfg["kappa"], x, rows_count, 1809_0002)
    pm, pmats = time_steps(pkg, torch, v, f, dict(cfg, m=info.m), pkg.DH2_MIXED, x_dev, 1, 0, stream)[0::2]
    pinfo = pmats[-1].get_info()
    fp64 = {}
    if with_fp64:
        # the plain FP64 form at the same order: the same accuracy class as the learned build
        x64 = torch.from_numpy(x).cuda()
        fm, fmats = time_steps(pkg, torch, v, f, dict(cfg, m=info.m), pkg.DH2_FP64, x64, 1, 0, stream)[0::2]
        fp64 = {"plain_fp64_same_order_build_s": float(np.mean(fm)) / 1e3,
                "plain_fp64_same_order_relerr": sampled_dense_error(pkg, torch, fmats[-1], ref_tree, cfg["kappa"], x,
                                                                    rows_count, 1809_0002)}
        fp64["speedup_learned_mixed_vs_fp64_same_order"] = fp64["plain_fp64_same_order_build_s"] / (
            float(np.mean(ms)) / 1e3)
        for m_ in fmats:
            m_.close()
    out = {"workload": cfg["workload"], "order_chosen": info.m, "configured_order": cfg["m"],
           "build_s": float(np.mean(ms)) / 1e3, "relerr_sampled_dense": err, "meets_eps": bool(err <= cfg["eps"]),
           "configured_order_relerr": err_configured,
           "configured_order_meets_eps": bool(err_configured <= cfg["eps"]),
           "rank_cap_retries": info.rank_cap_retries, "truncation_MB": info.truncation_bytes / 1e6,
           "plain_same_order_build_s": float(np.mean(pm)) / 1e3,
           "plain_same_order_truncation_MB": pinfo.truncation_bytes / 1e6, **fp64}
    for m_ in mats + pmats:
        m_.close()
    model.close()
    return out


BATCH_SEED = 1809_0003


def batch_measure(pkg, torch, count, stream):
    """The batched workload: `count` spheres/ellipsoids of 1280-20480 triangles
    (synth.batch_meshes), kappa U[4, 16], leaf 32, eta1 10, eta2 1, m 5, eps 1e-4.
    Builds are blocking host calls that fan out over several streams, so they are
    timed with the host clock around the call (trees included, built beforehand
    for the build-only figures); the products with CUDA events on `stream`, which
    joins the internal streams."""
    import synth

    meshes = synth.batch_meshes(count, BATCH_SEED)
    m, eta2, eta1, eps, leaf = 5, 1.0, 10.0, 1e-4, 32
    kappas = [k for _, _, k in meshes]
    ntri = int(sum(len(f) for _, f, _ in meshes))
    trees = [pkg.Tree(v, f, leaf_max=leaf) for v, f, _ in meshes]

    def batch_build(nstreams):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mats = pkg.build_batch(trees, kappas, m, eta2, eps, eta1=eta1, nstreams=nstreams, **TILES)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, mats

    _, warm = batch_build(8)             # warm-up: kernels loaded, pool sized
    for mt in warm:
        mt.close()
    t1, mats1 = batch_build(1)
    for mt in mats1:
        mt.close()
    t8, mats = batch_build(8)
    xs = [torch.from_numpy(synth.random_vector(len(f), BATCH_SEED + i)).to(torch.complex64).cuda()
          for i, (_, f, _) in enumerate(meshes)]
    ys = [torch.empty_like(x) for x in xs]

    def products(batched):
        if batched:
            pkg.matvec_batch(mats, xs, ys, stream)
        else:
            for mt, x, y in zip(mats, xs, ys):
                mt.matvec(x, y, stream)

    def mv_ms(batched, reps=5):
        for _ in range(2):
            products(batched)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            products(batched)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    mv_batch, mv_serial = mv_ms(True), mv_ms(False)
    mv_bytes = int(sum(mt.get_info().matvec_bytes for mt in mats))
    # end to end: host meshes in, trees + batched build
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trees2 = [pkg.Tree(v, f, leaf_max=leaf) for v, f, _ in meshes]
    mats2 = pkg.build_batch(trees2, kappas, m, eta2, eps, eta1=eta1, nstreams=8)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    for obj in mats + mats2 + trees + trees2:
        obj.close()
    return {"workload": f"batch{count}: spheres/ellipsoids (icosphere L3-L5, semi-axes U[0.5,2]^3 for half), "
                        f"kappa U[4,16], seed {BATCH_SEED}, leaf {leaf}, eta1 {eta1}, eta2 {eta2}, m {m}, eps {eps}",
            "meshes": count, "triangles": ntri,
            "build_s_8_streams": t8, "build_s_1_stream": t1, "build_speedup_streams": t1 / t8,
            "build_s_e2e_with_trees": t_e2e,
            "matvec_ms_batched": mv_batch, "matvec_ms_serial": mv_serial,
            "matvec_gbs_batched": mv_bytes / (mv_batch * 1e-3) / 1e9, "timing": "build: host clock around the "
            "blocking call; matvec: CUDA events on the joining stream"}


def max_over_ranks(values, torch, world, device):
    """Each value's maximum over the ranks (the slowest replica sets the step time); the
    values themselves when there is one rank.  device: "cuda" under NCCL, "cpu" under gloo."""
    if world <= 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = workload_config(args.workload)
    if args.m:
        cfg = dict(cfg, m=args.m, k=args.m ** 3)

    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        res = None
        for i in range(args.warmup + args.steps):
            res = run_oracle_child(args.workload)
            if i >= args.warmup:
                vals.append(res["value"])
        value = float(np.mean(vals))
        line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": 0, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(cfg, l2="inputs larger than L2"), "impl": "reference",
                "cpu_baseline": cpu_baseline_obj(dict(res, value=value)),
                "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch

    import paper_1809_04384_gb300 as pkg
    import synth

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    pkg.lib()
    precision = pkg.DH2_MIXED if args.precision == "mixed" else pkg.DH2_FP64
    v, f = workload_mesh(args.workload)
    n = len(f)
    x = synth.random_vector(n, 1809_0002)
    xdt = torch.complex64 if precision == pkg.DH2_MIXED else torch.complex128
    x_dev = torch.from_numpy(x).to(xdt).cuda()
    stream = torch.cuda.current_stream()
    main_model = pkg.Model.load() if args.learned else None

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    if args.qr_tpc:
        TILES.update(qr_tpc=tuple(int(t) for t in args.qr_tpc.split(",")), qr_group_rows=args.qr_group_rows)
        tuning = {"qr_threads_per_column": list(TILES["qr_tpc"]), "qr_group_rows": args.qr_group_rows,
                  "note": "fixed on the command line"}
    else:
        tuning = None if args.no_autotune else autotune(pkg, v, f, cfg, precision, stream)

    # warm-up and timed steps (one replica per GPU: the path is not sharded)
    launches0 = pkg.lib().dh2_kernel_launches()
    barrier()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        build_ms, mv_ms, mats = time_steps(pkg, torch, v, f, cfg, precision, x_dev, args.steps, args.warmup,
                                           stream, main_model)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    launches = pkg.lib().dh2_kernel_launches() - launches0
    launches_per_step = launches / (args.steps + args.warmup)
    build_s = float(np.mean(build_ms)) / 1e3
    step_ms = float(np.mean(np.array(build_ms) + np.array(mv_ms)))
    build_s, step_ms = max_over_ranks([build_s, step_ms], torch, world, "cuda")
    mat = mats[-1]
    info = mat.get_info()
    free_b, total_b = torch.cuda.mem_get_info()
    device_used_gb = (total_b - free_b) / 1e9

    # matvec throughput: algorithmic bytes / device time, repeated launches
    mv_rep_ms = matvec_repeat_ms(torch, mat, x_dev, 20, stream)
    mv_gbs = info.matvec_bytes / (mv_rep_ms * 1e-3) / 1e9

    # per-kernel device times summed over the timed builds
    ktimes = {}
    for m_ in mats:
        for name, (ms, cnt) in m_.kernel_times().items():
            a, b = ktimes.get(name, (0.0, 0))
            ktimes[name] = (a + ms, b + cnt)
    # matvec kernels with timing on
    mat.set_timing(True)
    for _ in range(10):
        mat.matvec(x_dev, torch.empty_like(x_dev), stream=stream)
    torch.cuda.synchronize()
    mv_kernels = {k: v_ for k, v_ in mat.kernel_times().items() if k.startswith("mv_")}
    mat.set_timing(False)
    work = kernel_work(mat, info, cfg)
    peaks = load_peaks()
    build_kernels = {k: v_ for k, v_ in ktimes.items() if not k.startswith("mv_") and v_[1] > 0}
    dom = max(build_kernels, key=lambda k: build_kernels[k][0])
    roof = roofline_obj(dom, build_kernels[dom], work, peaks, len(mats),
                        measured_traffic(cfg["workload"], dom, args.precision))
    leaf_ms, leaf_cnt = mv_kernels.get("mv_leaf_out", (0.0, 0))
    mv_roof = roofline_obj("mv_leaf_out", (leaf_ms, leaf_cnt), work, peaks, 10,
                           measured_traffic(cfg["workload"], "mv_leaf_out", args.precision))

    # e2e: host mesh in, host vector in/out, through the C ABI
    xh = np.ascontiguousarray(x.astype(np.complex128))
    e2e = []
    for i in range(0 if args.no_e2e else 1 + min(args.steps, 3)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = gpu_build(pkg, v, f, cfg, precision, None)
        m2.matvec_host(xh)
        torch.cuda.synchronize()
        if i > 0:
            e2e.append(time.perf_counter() - t0)
        m2.close()
    h2d = v.nbytes + f.astype(np.int32).nbytes + xh.nbytes
    d2h = xh.nbytes

    # accuracy against sampled dense rows (outside the timed region)
    ref_tree = pkg.Tree(v, f, leaf_max=cfg["leaf"])
    err = sampled_dense_error(pkg, torch, mat, ref_tree, cfg["kappa"], x, args.error_rows, 1809_0002)

    # plain FP64 GPU form of the same build
    fp64 = None
    if precision == pkg.DH2_MIXED and not args.no_fp64:
        x64 = torch.from_numpy(x).cuda()
        b64, m64, mats64 = time_steps(pkg, torch, v, f, cfg, pkg.DH2_FP64, x64, 2, 1, stream)
        mv64 = matvec_repeat_ms(torch, mats64[-1], x64, 10, stream)
        err64 = sampled_dense_error(pkg, torch, mats64[-1], ref_tree, cfg["kappa"], x, args.error_rows, 1809_0002)
        fp64 = {"build_s": float(np.mean(b64)) / 1e3, "matvec_ms": mv64,
                "matvec_gbs": mats64[-1].get_info().matvec_bytes / (mv64 * 1e-3) / 1e9,
                "matvec_relerr_sampled_dense": err64,
                "speedup_build_mixed_vs_fp64": float(np.mean(b64)) / 1e3 / build_s}
        for m_ in mats64:
            m_.close()

    learned = None
    if precision == pkg.DH2_MIXED and not args.no_learned and not args.learned:
        learned = learned_measure(pkg, torch, v, f, cfg, x, ref_tree, args.error_rows, err, stream,
                                  with_fp64=not args.no_fp64)

    batch = None
    if not args.no_batch:
        batch = batch_measure(pkg, torch, args.batch_meshes, stream)

    baseline = None
    if rank == 0 and not args.no_baseline:
        try:
            baseline = cpu_baseline_obj(run_oracle_child(args.workload))
        except Exception as e:  # reported, never silently replaced
            baseline = {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": build_s * world / world, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64" if precision == pkg.DH2_MIXED else "c128",
            "data": "synthetic",
            "config": dict(cfg, precision=args.precision, parallelism=f"replicas{world}",
                           order=("learned: " + str(info.m)) if args.learned else "configured",
                           l2="inputs larger than L2 (nearfield alone > 1 GB)"),
            "build_s": build_s,
            "matvec": {"gbs": mv_gbs, "ms": mv_rep_ms, "bytes": info.matvec_bytes,
                       "relerr_sampled_dense": err, "rows_sampled": args.error_rows,
                       "kernel_ms": {k: round(v_[0] / max(v_[1], 1) * (v_[1] / 10), 4)
                                     for k, v_ in mv_kernels.items()}},
            "ranks": {"max_row": info.max_rank_row, "mean_row": info.mean_rank_row,
                      "max_col": info.max_rank_col, "mean_col": info.mean_rank_col},
            "storage": {"near_entries": info.near_entries, "coupling_entries": info.coupling_entries,
                        "basis_entries": info.basis_entries, "nadm": info.nadm, "nnear": info.nnear},
            "stage_ms": {k: round(v_, 3) for k, v_ in mat.stage_ms().items()},
            "kernel_ms_per_step": {k: round(v_[0] / len(mats), 3) for k, v_ in build_kernels.items()},
            "roofline": roof,
            "matvec_roofline": mv_roof,
            "plain_fp64": fp64,
            "autotune": tuning,
            "learned": learned,
            "batch": batch,
            "cpu_baseline": baseline,
            "e2e": ({"value": float(np.mean(e2e)), "unit": "s", "h2d_bytes_per_step": int(h2d),
                     "d2h_bytes_per_step": int(d2h)} if e2e else None),
            "device_memory_used_gb": device_used_gb,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clk.summary(),
            "wall_s_timed_region": t_wall,
        }
        print(json.dumps(line))
    for m_ in mats:
        m_.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------------------- roofline

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], bf16=d["bf16_tflops"], sm_max_mhz=d.get("sm_max_mhz", 2070.0),
                    source="measured")
    return dict(hbm_gbs=6800.0, bf16=1900.0, sm_max_mhz=2070.0, source="fallback")


def kernel_work(mat, info, cfg):
    """Algorithmic work per kernel over one build / one matvec (library counters)."""
    return mat.kernel_work()


KERNEL_SOURCES = ["paper_1809_04384_gb300/csrc/numeric.cu", "paper_1809_04384_gb300/csrc/linalg.cuh",
                  "paper_1809_04384_gb300/csrc/common.cuh"]


def measured_traffic(workload, name, precision):
    """DRAM bytes per launch of kernel id `name` from the committed ncu summary of this
    workload, or None when there is none or the kernel sources changed since."""
    import hashlib

    path = os.path.join(ROOT, "profiles", f"dram_per_launch_{workload}_{precision}.txt")
    if not os.path.exists(path):
        return None
    text = open(path).read().split("\n")
    want = next((ln.split()[1] for ln in text if ln.startswith("sources_sha256_16:")), None)
    have = hashlib.sha256(b"".join(open(os.path.join(ROOT, p), "rb").read() for p in KERNEL_SOURCES)).hexdigest()[:16]
    if want != have:
        return None
    for ln in text:
        f = ln.split()
        if len(f) == 4 and f[0] == "traffic" and f[1] == workload and f[2] == name:
            return float(f[3])
    return None


def roofline_obj(name, timing, work, peaks, nsteps, traffic=None):
    ms, launches = timing
    if launches == 0 or ms <= 0:
        return None
    w = work.get(name)
    if w is None:
        return None
    kind, amount = w          # amount per build (or per matvec)
    per_launch_ms = ms / launches
    launches_per_step = launches / nsteps
    per_launch_work = amount / launches_per_step
    if kind == "byte":
        achieved = per_launch_work / (per_launch_ms * 1e-3) / 1e9
        peak = peaks["hbm_gbs"]
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peaks["source"] + " copy bandwidth",
                "algorithmic_bytes_per_launch": per_launch_work, "avg_launch_ms": per_launch_ms}
    # FP32 / FP64 SIMT arithmetic: peak from unit counts and the maximum SM clock
    lanes = {"flop32": 128, "flop64": 2}[kind]
    peak = 152 * lanes * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    achieved = per_launch_work / (per_launch_ms * 1e-3) / 1e12
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"derived: 152 SMs x {lanes} {'FP32' if lanes == 128 else 'FP64'} FMA lanes x 2 x "
                           f"{peaks['sm_max_mhz']:.0f} MHz",
            "algorithmic_flop_per_launch": per_launch_work, "avg_launch_ms": per_launch_ms}


if __name__ == "__main__":
    main()
