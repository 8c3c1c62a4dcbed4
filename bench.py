#!/usr/bin/env python
"""Benchmark of the GB300 hybrid DH^2 build + matvec.

One step = the whole hot path on one synthetic workload: cluster tree,
directions, block tree, nearfield, directional interpolation, basis weights,
total weights (rows and columns), SVD truncation, projection (dh2_build_tree +
dh2_build_dh2), then one DH^2 matvec (dh2_matvec).

Workload (default): unit sphere, icosahedral refinement to 20480 flat
triangles, kappa = 16 (kappa h ~ 0.5), leaf <= 32, eta1 = 10, eta2 = 1,
eps = 1e-4, seeded N(0,1) + i N(0,1) vectors; configured Chebyshev order m = 5
(k = 125).  The timed builds use the mixed form (complex FP32 kernel evaluation,
3xTF32 tensor-core products and FP32 storage; FP64 weight factorisations and
FP64 SVD truncation) and take their order from the shipped learned model
(`--order learned`, the default), which picks the order that meets eps on this
workload; `--order configured` or `--order N` fix it.

Prints ONE JSON line (rank 0).  `value` = build seconds per step (device time
with CUDA events on the launching stream).  Beside it: the matvec throughput
(algorithmic GB/s: every stored coefficient + the vectors, once) and the error of
the product on sampled rows against the FP64 Galerkin rows (dh2_dense_rows, every
column by quadrature on the GPU); side legs, each recorded as {"error": ...} if it
fails instead of ending the run: the configured order in the same form, the
all-FP32 variant and the plain FP64 form at the headline's order, a plain build at
the learned order, the 64-mesh batched build, the end-to-end time through the C ABI
with host buffers, and the CPU oracle on a bounded sample (`cpu_baseline`).
Only the last matrix of a leg stays on the device.  `--impl reference` times the
CPU oracle (the reference arm) on a bounded sample of the workload per step.

    python bench.py [--steps K] [--warmup W] [--form mixed|mixed32|fp64] [--order learned|configured|N]
                    [--impl ours|reference]
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
    ap.add_argument("--form", default="mixed", choices=["mixed", "mixed32", "fp64"],
                    help="mixed: FP32 products/storage with FP64 weight factorisations and SVD; "
                         "mixed32: all FP32; fp64: all FP64")
    ap.add_argument("--order", default="learned",
                    help="interpolation order of the timed builds: 'learned' (the shipped model chooses), "
                         "'configured' (the workload's m) or a number")
    ap.add_argument("--workload", default="sphere20480", choices=list(WORKLOADS))
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU form")
    ap.add_argument("--no-fp32", action="store_true", help="skip the all-FP32 variant")
    ap.add_argument("--error-rows", type=int, default=256)
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-mesh batched build")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end builds")
    ap.add_argument("--batch-meshes", type=int, default=64)
    ap.add_argument("--no-learned", action="store_true", help="skip the plain build at the learned order")
    ap.add_argument("--no-direct", action="store_true", help="skip the direct-recompression build")
    ap.add_argument("--no-dlp", action="store_true", help="skip the double-layer build")
    ap.add_argument("--m", type=int, default=0, help="override the workload's configured order")
    ap.add_argument("--no-autotune", action="store_true", help="library default tile shapes, no autotuning")
    ap.add_argument("--qr-tpc", default="", help="fixed FP32 weight-QR threads per column 'a,b,c' (skips autotuning)")
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

PATCH_LEVEL = 3   # the sampled patch: the triangles under one cluster of this tree level


def oracle_sample_seconds(name, out_queue=None):
    """Times the oracle on a bounded sample of the workload (runs in a child process).

    Sample: the full structure phase (cluster tree, directions, block tree) of the
    workload, plus the complete build (nearfield + interpolation + recompression) of
    the mesh patch under one cluster of level PATCH_LEVEL (same mesh density, kappa,
    leaf, m, eps).  `sample_seconds` is what the oracle ran; `estimate_s` scales the
    patch costs to the full workload by its admissible-block and nearfield-entry counts.
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
    plevel = min(PATCH_LEVEL, tr.depth)
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
    Recompression(dh, eps)
    t2 = time.perf_counter()
    for (a, b) in b2.near:
        dh.nearfield_block(a, b)
    t3 = time.perf_counter()
    near_s = int(sum(tr2.size[a] * tr2.size[b] for a, b in b2.near))
    t_recomp = t2 - t1
    t_near = t3 - t2
    est = t_struct + t_recomp * nadm_full / max(len(b2.adm), 1) + t_near * near_full / max(near_s, 1)
    return dict(estimate_s=est, sample_seconds=t_struct + (t3 - t0), patch_triangles=len(fs), patch_level=plevel,
                patch_adm=len(b2.adm), patch_near_entries=near_s, full_adm=nadm_full, full_near_entries=near_full,
                t_struct=t_struct, t_recomp=t_recomp, t_near=t_near)


def oracle_full_small_seconds():
    """The complete oracle (structure, nearfield, interpolation, recompression, one matvec)
    on the 1280-triangle sphere with the paper's parameters (kappa 4, leaf 32, m 4)."""
    import synth
    from oracle.geometry import Discretisation
    from oracle.interp import InterpolatedDH2
    from oracle.recompress import Recompression
    from oracle.structure import build_block_tree, build_cluster_tree, build_directions

    (_, lev), kappa, leaf, eta1, eta2, m, eps = WORKLOADS["sphere1280"]
    v, f = synth.icosphere(lev)
    x = synth.random_vector(len(f), 1809_0001)
    t0 = time.perf_counter()
    tr = build_cluster_tree(v, f, leaf)
    dirs = build_directions(tr, kappa, eta1)
    bt = build_block_tree(tr, dirs, kappa, eta2)
    dh = InterpolatedDH2(Discretisation(v, f), tr, dirs, bt, kappa, m)
    rc = Recompression(dh, eps)
    t1 = time.perf_counter()
    rc.matvec(x)
    t2 = time.perf_counter()
    return dict(workload="icosphere1280 (kappa 4, leaf 32, m 4; no admissible block: the nearfield is all of G)",
                build_s=t1 - t0, build_includes="structure, interpolation, recompression",
                matvec_s=t2 - t1, matvec_includes="the oracle's product, which evaluates the nearfield blocks",
                triangles=len(f))


def run_oracle_child(func, *args):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.%s(*%r)))" % (ROOT, func, tuple(args)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def sample_text(res):
    return (f"oracle structure phase on the full mesh + complete oracle build (nearfield, interpolation, "
            f"recompression) of a {res['patch_triangles']}-triangle patch (one level-{res['patch_level']} "
            f"cluster) of the same mesh, single-threaded")


def estimate_text(res):
    return (f"structure + recompression x (admissible blocks {res['full_adm']} / {res['patch_adm']}) + nearfield x "
            f"(entries {res['full_near_entries']} / {res['patch_near_entries']})")


def cpu_baseline_obj(res):
    """The oracle's full-workload build time is an estimate from a measured sample."""
    return {"value": res["estimate_s"], "unit": "s", "cores": 1, "kind": "oracle", "estimate": True,
            "estimate_formula": estimate_text(res), "sample": sample_text(res),
            "sample_seconds_measured": res["sample_seconds"]}


# ----------------------------------------------------------------------------- GPU arm

TILES = {}   # FP32 weight-QR tile shapes chosen by the autotuner for this run (empty: library defaults)


def gpu_build(pkg, v, f, cfg, form, stream, model=None, **extra):
    """Tree + DH^2 build of one workload.  form: 'mixed' (FP32 products and storage, FP64
    weight factorisations and SVD), 'mixed32' (all FP32) or 'fp64'.  extra: further Matrix
    options (e.g. direct=1)."""
    tree = pkg.Tree(v, f, leaf_max=cfg["leaf"], stream=stream)
    prec = pkg.DH2_FP64 if form == "fp64" else pkg.DH2_MIXED
    f64 = 0 if form == "mixed32" else 1
    mat = pkg.Matrix(tree, cfg["kappa"], cfg["m"], cfg["eta2"], cfg["eps"], precision=prec, eta1=cfg["eta1"],
                     qr_fp64=f64, svd_fp64=f64, model=model, stream=stream, **(TILES if form == "mixed32" else {}),
                     **extra)
    tree.close()
    return mat


def release(pkg, torch):
    """Returns cached device memory of both allocators between the legs."""
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    pkg.dh2_release_cached()


def autotune(pkg, v, f, cfg, stream):
    """dh2_autotune of the FP32 weight-QR tiles on the workload itself (outside the timed region);
    the all-FP32 builds of the run use them."""
    tree = pkg.Tree(v, f, leaf_max=cfg["leaf"], stream=stream)
    base = pkg.options(eta1=cfg["eta1"], precision=pkg.DH2_MIXED, qr_fp64=0, svd_fp64=0)
    t0 = time.perf_counter()
    tuned, t_ms, b_ms = pkg.dh2_autotune(tree.handle, cfg["kappa"], cfg["m"], cfg["eta2"], cfg["eps"], base, reps=2,
                                         stream=stream)
    wall = time.perf_counter() - t0
    tree.close()
    TILES.update(qr_tpc=tuple(int(t) for t in tuned.qr_tpc), qr_group_rows=int(tuned.qr_group_rows))
    return {"qr_threads_per_column": list(TILES["qr_tpc"]), "qr_group_rows": TILES["qr_group_rows"],
            "qr_ms_per_build_tuned": t_ms, "qr_ms_per_build_default": b_ms, "tuning_s": wall, "applies_to": "mixed32",
            "note": "0 = library default (8, 4, 2 threads per column; 1024-row groups)"}


def time_steps(pkg, torch, v, f, cfg, form, x_dev, steps, warmup, stream, model=None, **extra):
    """Device-timed steps: build (tree + DH^2) and one matvec, CUDA events on `stream`.
    Only the last matrix is kept (returned open); the per-kernel and per-stage device
    times of the timed builds are summed as they go."""
    build_ms, mv_ms = [], []
    ktot, stot = {}, {}
    last = None
    for i in range(warmup + steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        y = torch.empty_like(x_dev)
        torch.cuda.synchronize()
        e0.record(stream)
        mat = gpu_build(pkg, v, f, cfg, form, stream, model, **extra)
        e1.record(stream)
        mat.matvec(x_dev, y, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            build_ms.append(e0.elapsed_time(e1))
            mv_ms.append(e1.elapsed_time(e2))
            for name, (ms, cnt) in mat.kernel_times().items():
                a, b = ktot.get(name, (0.0, 0))
                ktot[name] = (a + ms, b + cnt)
            for name, ms in mat.stage_ms().items():
                stot[name] = stot.get(name, 0.0) + ms
        if last is not None:
            last.close()
        last = mat
    return build_ms, mv_ms, ktot, stot, last


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


ERROR_SEED = 1809_0002


def error_rows(n, count, seed=ERROR_SEED):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(count, n), replace=False))


def sampled_dense_error(pkg, torch, mat, ref, rows, x):
    """Relative 2-norm error of the product on sampled rows against the FP64 Galerkin rows
    `ref` (dh2_dense_rows: every column by quadrature, on the GPU)."""
    dt = torch.complex64 if mat.precision == pkg.DH2_MIXED else torch.complex128
    y = mat.matvec(torch.from_numpy(x).to(dt).cuda()).cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref))


def side_build(pkg, torch, v, f, cfg, form, x, ref, rows, stream, model=None, steps=2, **extra):
    """One warm-up and `steps` timed builds of a variant; its product error and sizes."""
    x_dev = torch.from_numpy(x).to(torch.complex128 if form == "fp64" else torch.complex64).cuda()
    b, mv, kt, _, mat = time_steps(pkg, torch, v, f, cfg, form, x_dev, steps, 1, stream, model, **extra)
    info = mat.get_info()
    mv_ms = matvec_repeat_ms(torch, mat, x_dev, 10, stream)
    out = {"form": form, "m": info.m, "build_s": float(np.mean(b)) / 1e3,
           "relerr_sampled_dense": (sampled_dense_error(pkg, torch, mat, ref, rows, x) if ref is not None
                                    else None),
           "matvec_ms": mv_ms, "matvec_gbs": info.matvec_bytes / (mv_ms * 1e-3) / 1e9,
           "truncation_MB": info.truncation_bytes / 1e6, "rank_cap_retries": info.rank_cap_retries,
           "peak_pool_GB": info.peak_pool_bytes / 1e9, "symmetric": info.symmetric,
           "kernel_ms_per_build": {k: round(a / steps, 2) for k, (a, c) in kt.items() if c}}
    if ref is not None:
        out["meets_eps"] = bool(out["relerr_sampled_dense"] <= cfg["eps"])
    out["mean_rank_row"], out["mean_rank_col"] = info.mean_rank_row, info.mean_rank_col
    mat.close()
    return out


BATCH_SEED = 1809_0003


def batch_measure(pkg, torch, count, stream, form="mixed"):
    """The batched workload: `count` spheres/ellipsoids of 1280-20480 triangles
    (synth.batch_meshes), kappa U[4, 16], leaf 32, eta1 10, eta2 1, m 5, eps 1e-4.
    Builds are blocking host calls that fan out over several streams, so they are
    timed with the host clock around the call (trees built beforehand for the
    build-only figures); the products with CUDA events on `stream`, which joins the
    internal streams.  Every batch of matrices is freed before the next is built."""
    import synth

    meshes = synth.batch_meshes(count, BATCH_SEED)
    m, eta2, eta1, eps, leaf = 5, 1.0, 10.0, 1e-4, 32
    f64 = 0 if form == "mixed32" else 1
    kappas = [k for _, _, k in meshes]
    ntri = int(sum(len(f) for _, f, _ in meshes))
    trees = [pkg.Tree(v, f, leaf_max=leaf) for v, f, _ in meshes]
    tiles = TILES if form == "mixed32" else {}

    def batch_build(nstreams, trs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mats = pkg.build_batch(trs, kappas, m, eta2, eps, eta1=eta1, nstreams=nstreams, qr_fp64=f64, svd_fp64=f64,
                               **tiles)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, mats

    def close_all(objs):
        for o in objs:
            o.close()

    _, warm = batch_build(8, trees)      # warm-up: kernels loaded, pool sized
    close_all(warm)
    t1, mats1 = batch_build(1, trees)
    close_all(mats1)
    t8, mats = batch_build(8, trees)
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
    close_all(mats)
    close_all(trees)
    del xs, ys
    release(pkg, torch)
    # end to end: host meshes in, trees + batched build
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trees2 = [pkg.Tree(v, f, leaf_max=leaf) for v, f, _ in meshes]
    _, mats2 = batch_build(8, trees2)
    t_e2e = time.perf_counter() - t0
    close_all(mats2)
    close_all(trees2)
    return {"workload": f"batch{count}: spheres/ellipsoids (icosphere L3-L5, semi-axes U[0.5,2]^3 for half), "
                        f"kappa U[4,16], seed {BATCH_SEED}, leaf {leaf}, eta1 {eta1}, eta2 {eta2}, m {m}, eps {eps}",
            "form": form, "meshes": count, "triangles": ntri,
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


def leg(results, name, fn):
    """Runs one side measurement; a failure is recorded in the line instead of ending the run."""
    t0 = time.perf_counter()
    try:
        results[name] = fn()
    except Exception as e:   # recorded, never silently replaced
        results[name] = {"error": f"{type(e).__name__}: {e}"[:500]}
    if isinstance(results[name], dict):
        results[name]["leg_wall_s"] = round(time.perf_counter() - t0, 2)


FORMS = {"mixed": "c64+f64 (complex FP32 kernel evaluation, 3xTF32 tensor-core products and storage; "
                  "FP64 weight factorisations and SVD truncation)",
         "mixed32": "c64 (complex FP32 everywhere: products, weight QRs, SVD truncation)",
         "fp64": "c128 (complex FP64 everywhere)"}
DTYPES = {"mixed": "c64+f64", "mixed32": "c64", "fp64": "c128"}


def reference_arm(args, cfg):
    """The CPU oracle on a bounded sample of the workload per step (rank 0 only)."""
    samples = []
    res = None
    for i in range(args.warmup + args.steps):
        res = run_oracle_child("oracle_sample_seconds", args.workload)
        if i >= args.warmup:
            samples.append(res)
    value = float(np.mean([r["sample_seconds"] for r in samples]))
    est = float(np.mean([r["estimate_s"] for r in samples]))
    try:
        small = run_oracle_child("oracle_full_small_seconds")
    except Exception as e:
        small = {"error": str(e)[:500]}
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, l2="inputs larger than L2", sample=sample_text(res)), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample_text(res)},
            "full_workload_estimate_s": est, "full_workload_estimate_formula": estimate_text(res),
            "oracle_full_icosphere1280": small,
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = workload_config(args.workload)
    if args.m:
        cfg = dict(cfg, m=args.m, k=args.m ** 3)

    if args.impl == "reference":
        if rank == 0:
            reference_arm(args, cfg)
        return

    import torch

    import paper_1809_04384_gb300 as pkg
    import synth

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    pkg.lib()
    form = args.form
    v, f = workload_mesh(args.workload)
    n = len(f)
    x = synth.random_vector(n, ERROR_SEED)
    xdt = torch.complex128 if form == "fp64" else torch.complex64
    x_dev = torch.from_numpy(x).to(xdt).cuda()
    stream = torch.cuda.current_stream()
    model = pkg.Model.load() if args.order == "learned" else None
    if args.order not in ("learned", "configured"):
        cfg = dict(cfg, m=int(args.order), k=int(args.order) ** 3)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    side = {}

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # FP32 weight-QR tiles for the all-FP32 builds (outside the timed region)
    if args.qr_tpc:
        TILES.update(qr_tpc=tuple(int(t) for t in args.qr_tpc.split(",")), qr_group_rows=args.qr_group_rows)
        side["autotune"] = {"qr_threads_per_column": list(TILES["qr_tpc"]), "qr_group_rows": args.qr_group_rows,
                            "note": "fixed on the command line"}
    elif not args.no_autotune:
        leg(side, "autotune", lambda: autotune(pkg, v, f, cfg, stream))

    # warm-up and timed steps (one replica per GPU: the path is not sharded)
    launches0 = pkg.lib().dh2_kernel_launches()
    barrier()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        build_ms, mv_ms, ktimes, stimes, mat = time_steps(pkg, torch, v, f, cfg, form, x_dev, args.steps,
                                                          args.warmup, stream, model)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    launches = pkg.lib().dh2_kernel_launches() - launches0
    launches_per_step = launches / (args.steps + args.warmup)
    build_s = float(np.mean(build_ms)) / 1e3
    step_ms = float(np.mean(np.array(build_ms) + np.array(mv_ms)))
    build_s, step_ms = max_over_ranks([build_s, step_ms], torch, world, "cuda")
    info = mat.get_info()
    order = info.m
    cfg_run = dict(cfg, m=order, k=order ** 3)
    free_b, total_b = torch.cuda.mem_get_info()
    device_used_gb = (total_b - free_b) / 1e9

    # matvec throughput: algorithmic bytes / device time, repeated launches
    mv_rep_ms = matvec_repeat_ms(torch, mat, x_dev, 20, stream)
    mv_gbs = info.matvec_bytes / (mv_rep_ms * 1e-3) / 1e9
    mat.set_timing(True)
    for _ in range(10):
        mat.matvec(x_dev, torch.empty_like(x_dev), stream=stream)
    torch.cuda.synchronize()
    mv_kernels = {k: v_ for k, v_ in mat.kernel_times().items() if k.startswith("mv_")}
    mat.set_timing(False)
    work = mat.kernel_work()
    peaks = load_peaks(sms)
    build_kernels = {k: v_ for k, v_ in ktimes.items() if not k.startswith("mv_") and v_[1] > 0}
    dom = max(build_kernels, key=lambda k: build_kernels[k][0])
    roof = roofline_obj(dom, build_kernels[dom], work, peaks, args.steps,
                        measured_traffic(cfg["workload"], dom, form))
    # every build kernel against its own bound (compact: bound, achieved, unit, frac)
    kernel_roofs = {}
    for kname in sorted(build_kernels):
        r = roofline_obj(kname, build_kernels[kname], work, peaks, args.steps)
        if r is not None:
            kernel_roofs[kname] = {"bound": r["bound"], "achieved": round(r["achieved"], 3), "unit": r["unit"],
                                   "frac": round(r["frac"], 4)}
    leaf_ms, leaf_cnt = mv_kernels.get("mv_leaf_out", (0.0, 0))
    mv_roof = roofline_obj("mv_leaf_out", (leaf_ms, leaf_cnt), work, peaks, 10,
                           measured_traffic(cfg["workload"], "mv_leaf_out", form))

    # accuracy against sampled dense rows (outside the timed region)
    rows = error_rows(n, args.error_rows)
    ref_tree = pkg.Tree(v, f, leaf_max=cfg["leaf"])
    ref = pkg.dh2_dense_rows(ref_tree.handle, cfg["kappa"], rows, torch.from_numpy(x).cuda())
    ref_tree.close()
    err = sampled_dense_error(pkg, torch, mat, ref, rows, x)
    minfo = {"gbs": mv_gbs, "ms": mv_rep_ms, "bytes": info.matvec_bytes, "relerr_sampled_dense": err,
             "rows_sampled": len(rows),
             "kernel_ms": {k: round(v_[0] / max(v_[1], 1) * (v_[1] / 10), 4) for k, v_ in mv_kernels.items()}}
    headline = {
        "ranks": {"max_row": info.max_rank_row, "mean_row": info.mean_rank_row,
                  "max_col": info.max_rank_col, "mean_col": info.mean_rank_col},
        "storage": {"near_entries": info.near_entries, "coupling_entries": info.coupling_entries,
                    "basis_entries": info.basis_entries, "nadm": info.nadm, "nnear": info.nnear},
        "stage_ms_per_build": {k: round(v_ / args.steps, 3) for k, v_ in stimes.items()},
        "kernel_ms_per_build": {k: round(v_[0] / args.steps, 3) for k, v_ in build_kernels.items()},
        "truncation_MB": info.truncation_bytes / 1e6, "rank_cap_retries": info.rank_cap_retries,
        "peak_pool_GB": info.peak_pool_bytes / 1e9, "symmetric": info.symmetric,
    }
    mat.close()
    release(pkg, torch)

    # e2e: host mesh in, host vector in/out, through the C ABI, copies inside the timed region
    def e2e_leg():
        xh = np.ascontiguousarray(x.astype(np.complex128))
        times = []
        for i in range(1 + min(args.steps, 3)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m2 = gpu_build(pkg, v, f, cfg, form, None, model)
            m2.matvec_host(xh)
            torch.cuda.synchronize()
            if i > 0:
                times.append(time.perf_counter() - t0)
            m2.close()
        return {"value": float(np.mean(times)), "unit": "s",
                "h2d_bytes_per_step": int(v.nbytes + f.astype(np.int32).nbytes + xh.nbytes),
                "d2h_bytes_per_step": int(xh.nbytes)}

    if not args.no_e2e:
        leg(side, "e2e", e2e_leg)
        release(pkg, torch)
    # the configured order of the workload in the same form (reported beside the headline order)
    if args.order != "configured" and order != WORKLOADS[args.workload][5]:
        leg(side, "configured_order", lambda: side_build(pkg, torch, v, f, dict(cfg, m=WORKLOADS[args.workload][5]),
                                                         form, x, ref, rows, stream))
        release(pkg, torch)
    if form != "mixed32" and not args.no_fp32:
        leg(side, "all_fp32", lambda: side_build(pkg, torch, v, f, cfg_run, "mixed32", x, ref, rows, stream))
        release(pkg, torch)
    if form != "fp64" and not args.no_fp64:
        leg(side, "plain_fp64", lambda: side_build(pkg, torch, v, f, cfg_run, "fp64", x, ref, rows, stream))
        release(pkg, torch)
    if model is not None and not args.no_learned:
        leg(side, "plain_same_order", lambda: side_build(pkg, torch, v, f, cfg_run, form, x, ref, rows, stream))
        release(pkg, torch)
    if not args.no_dlp:
        # the double layer operator on the same mesh and order (no dense reference rows: its
        # error is checked against the oracle in the tests)
        leg(side, "double_layer", lambda: side_build(pkg, torch, v, f, cfg_run, form, x, None, rows, stream,
                                                     layer=pkg.DH2_DOUBLE_LAYER))
        release(pkg, torch)
    if not args.no_direct:
        leg(side, "direct_recompression", lambda: side_build(pkg, torch, v, f, cfg_run, form, x, ref, rows, stream,
                                                             direct=1))
        release(pkg, torch)
    if not args.no_batch:
        leg(side, "batch", lambda: batch_measure(pkg, torch, args.batch_meshes, stream, form))
        release(pkg, torch)
    if rank == 0 and not args.no_baseline:
        leg(side, "cpu_baseline", lambda: cpu_baseline_obj(run_oracle_child("oracle_sample_seconds", args.workload)))

    pf = side.get("plain_fp64", {})
    if "build_s" in pf:
        pf["speedup_build_vs_fp64"] = pf["build_s"] / build_s
    if rank == 0:
        e2e = side.pop("e2e", None)
        line = {
            "metric": METRIC, "value": build_s, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[form], "data": "synthetic",
            "config": dict(cfg_run, precision=FORMS[form], parallelism=f"replicas{world}",
                           order=(f"learned model: m = {order}" if model is not None else f"m = {order}"),
                           configured_order=WORKLOADS[args.workload][5],
                           l2="inputs larger than L2 (nearfield alone > 1 GB)"),
            "build_s": build_s, "meets_eps": bool(err <= cfg["eps"]),
            "matvec": minfo, **headline,
            "roofline": roof,
            "matvec_roofline": mv_roof,
            "build_kernel_rooflines": kernel_roofs,
            **{k: side.get(k) for k in ("configured_order", "all_fp32", "plain_fp64", "plain_same_order",
                                         "direct_recompression", "double_layer", "batch", "autotune")},
            "cpu_baseline": side.get("cpu_baseline"),
            "e2e": (e2e if e2e and "value" in e2e else {"error": (e2e or {}).get("error", "not run")}),
            "device_memory_used_gb": device_used_gb, "sm_count": sms,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clk.summary(),
            "wall_s_timed_region": t_wall,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------------------- roofline

def load_peaks(sms=152):
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], bf16=d["bf16_tflops"], sm_max_mhz=d.get("sm_max_mhz", 2070.0),
                    source="measured", sms=sms)
    return dict(hbm_gbs=6800.0, bf16=1900.0, sm_max_mhz=2070.0, source="fallback", sms=sms)


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
    if kind == "tc_bf16":   # BF16 tensor-core products (the integer-digit Gram): the measured BF16 peak
        achieved = per_launch_work / (per_launch_ms * 1e-3) / 1e12
        peak = peaks["bf16"]
        return {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": peaks["source"] + " dense BF16 (cuBLAS, burst)",
                "algorithmic_flop_per_launch": per_launch_work, "avg_launch_ms": per_launch_ms}
    # FP32 / FP64 SIMT arithmetic: peak from unit counts (FMA per SM per clock) and the maximum SM clock
    lanes = {"flop32": 128, "flop64": 2}[kind]
    sms = peaks.get("sms", 152)
    peak = sms * lanes * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    achieved = per_launch_work / (per_launch_ms * 1e-3) / 1e12
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"derived: {sms} SMs (device properties) x {lanes} {'FP32' if lanes == 128 else 'FP64'} "
                           f"FMA per SM per clock x 2 flop x {peaks['sm_max_mhz']:.0f} MHz",
            "algorithmic_flop_per_launch": per_launch_work, "avg_launch_ms": per_launch_ms}


if __name__ == "__main__":
    main()
