#!/usr/bin/env python
"""Benchmark of the rasterizer hot path: one step = one batched training step (preprocess,
binning, forward blend, L1 loss, backward blend, preprocess backward) over 16 views of
1280x832 of a 1M-Gaussian masked scene (64 blobs + 10% shell, SH degree 3, volume and
SH-band masks at eps = 0.5).

Prints one JSON line. value = views per second of the batched step with inputs resident in
HBM; e2e = the same through one C-ABI call per step with the Gaussian parameters and target
images in pinned host memory (tgs_train_step_batched_host: the library copies them in, the
copies of a step overlapping the compute of the steps before it, and copies the loss back).
Also reports the plain single-view path (views/s, at tile 16 and at its best configuration)
and forward-only render FPS for comparison, a significance pruning round, the roofline of the
dominant kernel against peaks measured on the GPU (tgs_measure_peaks), a sub-record for each of
the other four workloads (10K plain, 500K mixed-resolution batch, 300K render-only at
1920x1080, 3M large scene), and the FP64 CPU oracle timed on the host cores on a bounded
sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torchrun: every rank renders its own 16 views (replicas; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GAUSS = 1_000_000
N_VIEWS = 16
W, H = 1280, 832
METRIC = "fwd+bwd views/sec @1M Gaussians 1280x832 (batched step)"
# float32 operations per (pixel, fragment) pair, counted from blend_common.cuh:
OPS_EVAL = 11        # offset, exponent, skip tests, ex2, alpha: every evaluated pair (forward)
OPS_BLEND = 7        # 1 - a, T update, stop test, weight, 3 colour FMAs: contributing pairs
OPS_BWD = 51         # evaluation again + T recovery, colour-behind update, dL/da and the 9
                     # gradient terms: contributing pairs (skipped pairs not counted)
# special-function operations per contributing pair: ex2 in the forward, ex2 and the
# reciprocal of the T recovery in the backward
SFU_PER_CONTRIB = 3
# DRAM bytes (read + write) of one fused-blend launch (k_fused_warp) on the default workload at
# tile 32, 2 px/thread, batch 1, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum;
# the command is in profiles/k_fused_warp_300k_8x1280x832_tile32_ppt2.md). Reported only while the
# kernel's sources, its launcher included, are the ones measured (their sha256 below), else null.
FUSED_TRAFFIC = {"bytes": 633241344 + 87551744, "tile": 32, "ppt": 2, "batch": 1,
                 "sources": ("fused.cu", "blend_warp.cuh", "blend_common.cuh", "tgs_internal.cuh"),
                 "sha256": "bb6aba3e8d5a8e06da9626496de4269e41839415df1e7b73cdaff3a9cb61cfd5"}


def fused_traffic(cfg, n, views):
    import hashlib
    t = FUSED_TRAFFIC
    if (cfg.tile, cfg.ppt, max(cfg.batch, 1), n, views) != (t["tile"], t["ppt"], t["batch"], N_GAUSS, N_VIEWS):
        return None
    h = hashlib.sha256()
    for f in t["sources"]:
        with open(os.path.join(ROOT, "paper_2501_14534_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return t["bytes"] if h.hexdigest() == t["sha256"] else None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_GAUSS)
    p.add_argument("--views", type=int, default=N_VIEWS)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-workloads", action="store_true",
                   help="skip the sub-records of the 10K, 500K, 300K and 3M workloads")
    p.add_argument("--no-pruning-round", action="store_true")
    p.add_argument("--tile", type=int, default=16)
    p.add_argument("--ppt", type=int, default=1)
    p.add_argument("--step-only", action="store_true",
                   help="stop after the timed batched steps (for launch lists under a profiler)")
    return p.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(n, views, seed_offset=0):
    from paper_2501_14534_gb300 import synth
    w = synth.workload(2, n=n, n_views=views)
    return w


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist(per_ms):
    """Median, p10 and p90 of per-step times (ms)."""
    a = np.asarray(per_ms, np.float64)
    return {"median": float(np.median(a)), "p10": float(np.percentile(a, 10)),
            "p90": float(np.percentile(a, 90))}


def timed(torch, fn, steps, stream):
    """Runs fn steps times back to back on stream with an event after each; returns the total
    and the per-step times in ms."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for i in range(steps):
            fn()
            ev[i + 1].record(stream)
    stream.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[-1]), per


# ---- algorithmic work and the floor of a step (the roofline of the whole path) ----------
#
# bytes / ops per unit as stated in the design doc: preprocess reads each Gaussian's 252 B once for
# all views and writes a 48 B record per (view, Gaussian); binning scans 8 B per record and
# moves 12 B per key written plus 24 B per key per 8-bit sort pass over 32 depth bits and the
# tile bits, and reads 8 B per key for the ranges; the blend is bound by FP32 issue (ops per
# pair above) or the SFU (SFU_PER_CONTRIB per contributing pair), whichever is slower, plus
# 40 B per key gathered; the preprocess backward reads 252 B and writes 252 B + 12 B of
# statistics per Gaussian and reads 36 B per (view, Gaussian).

def key_passes(total_tiles):
    return (32 + max(1, int(np.ceil(np.log2(max(total_tiles, 2))))) + 7) // 8


def step_floor_ms(n, V, K, tiles, pixels, P_eval, P_contrib, peaks, hbm_gbs, backward=True, gbytes_param=252):
    """Per-stage floors (ms) of one step from its algorithmic work and the measured peaks."""
    hbm = hbm_gbs * 1e9
    fp32 = peaks["fp32_fma_per_s"]
    sfu = peaks["ex2_per_s"]
    st = {}
    st["preprocess"] = (gbytes_param * n + 48 * V * n) / hbm * 1e3
    st["binning"] = (8 * V * n + K * (12 + 24 * key_passes(tiles) + 8)) / hbm * 1e3
    ops = P_eval * OPS_EVAL + P_contrib * OPS_BLEND + (P_contrib * OPS_BWD if backward else 0)
    sfu_ops = P_contrib * (SFU_PER_CONTRIB if backward else 1)
    gather = (40 * K * (2 if backward else 1) + (24 if backward else 12) * pixels) / hbm
    st["blend"] = max(ops / fp32, sfu_ops / sfu, gather) * 1e3
    if backward:
        st["preprocess_backward"] = ((252 + 252 + 12) * n + 36 * V * n) / hbm * 1e3
    return st


def pair_counts(R, g, cams, tile, ppt, eps_mask, eps_sh):
    """Exact (pixel, fragment) pair counts of these views at this tile size, from a forward
    with per-pixel counters: evaluated (pixel in the splat's rect, before the pixel stopped)
    and contributing (blended)."""
    counter = R.Rasterizer(tile=tile, ppt=ppt, eps_mask=eps_mask, eps_sh=eps_sh)
    Pe = Pc = 0
    for c in cams:
        o = counter.forward(g, [c], want_examined=True, want_counts=True)[0]
        Pe += int(o["n_eval"].sum().item())
        Pc += int(o["n_contrib"].sum().item())
    return Pe, Pc


def cpu_baseline(w, fraction=1.0 / 64, threads=None):
    """The FP64 oracle on the host cores for ONE view: preprocess, key sort, forward blend,
    L1 loss, backward blend and preprocess backward. The per-tile blend work (forward and
    backward) runs on an evenly spaced sample of the tiles, over the lists of the full key
    sort, and is scaled to all tiles; everything else runs in full.
    Returns (views/s, cores, description, seconds of CPU work)."""
    import oracle
    cores = threads or len(os.sched_getaffinity(0))
    sc, cam, tgt = w["scene"], w["cams"][0], w["targets"][0]
    st = oracle.Settings(tile=16, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    t0 = time.perf_counter()
    sp = oracle.preprocess(sc, cam, st)
    t_pre = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, vals, ranges = oracle.keys(sp["radius"], sp["rect"], sp["depth"], cam.width, cam.height, 16)
    t_keys = time.perf_counter() - t0
    T = ranges.shape[0]
    step = max(1, int(round(1.0 / fraction)))
    mask = np.zeros(T, np.uint8)
    mask[::step] = 1
    f = mask.sum() / T
    t0 = time.perf_counter()
    out = oracle.blend(sp, cam.width, cam.height, 16, tile_mask=mask, nthreads=cores,
                       lists=(vals, ranges))
    t_fwd = time.perf_counter() - t0
    _, dls = oracle.l1([out["image"]], [tgt])
    t0 = time.perf_counter()
    g9 = oracle.blend_backward(sp, cam.width, cam.height, dls[0], 16, nthreads=cores,
                               tile_mask=mask, lists=(vals, ranges))
    t_bwd = time.perf_counter() - t0
    grads = oracle.zero_grads(sc)
    t0 = time.perf_counter()
    oracle.preprocess_backward(sc, cam, st, g9, grads, oracle.new_stats(g9.shape[0]))
    t_pbwd = time.perf_counter() - t0
    t_view = t_pre + t_keys + (t_fwd + t_bwd) / f + t_pbwd
    sample_s = t_pre + t_keys + t_fwd + t_bwd + t_pbwd
    desc = (f"1 view of {sc['means'].shape[0]} Gaussians at {cam.width}x{cam.height}: preprocess, "
            f"key sort and preprocess backward in full; forward and backward blend on "
            f"{int(mask.sum())} of {T} tiles (every {step}th) scaled to all tiles; "
            f"{sample_s:.1f} s of CPU work on {cores} threads")
    return 1.0 / t_view, cores, desc, sample_s


def run_reference(args, rank, world):
    """The oracle as the reference arm, on the host cores (rank 0 only)."""
    if rank != 0:
        return
    full = workload(args.n, args.views)
    w = dict(full, cams=full["cams"][:1], targets=full["targets"][:1])   # one view per step
    # size the per-step sample so that warmup + steps end within about three minutes
    budget = 170.0 / max(1, args.steps + args.warmup)
    fraction = 1.0 / 64
    vals = []
    for i in range(args.warmup + args.steps):
        v, cores, desc, took = cpu_baseline(w, fraction)
        if i >= args.warmup:
            vals.append(v)
        if took > budget and fraction > 1.0 / 4096:
            fraction /= 2.0
    value = float(np.median(vals))
    line = {"metric": METRIC, "value": value, "unit": "views/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": full["name"], "global_batch": len(full["cams"]),
                       "views_per_gpu": len(full["cams"]), "inputs": "host memory",
                       "sample": "each step: the first view of the workload, in part (see cpu_baseline)"},
            "cpu_baseline": {"value": value, "unit": "views/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "views/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- the other workloads ------------------------------------------------------------------

def _floor_record(st_ms, measured_ms):
    floor = sum(st_ms.values())
    return {"bound": "step", "floor_ms": floor, "measured_ms": measured_ms, "frac": floor / measured_ms,
            "stage_floor_ms": st_ms,
            "note": "sum of the stage floors (HBM stages at the measured copy bandwidth, blend at the "
                    "measured FP32 issue / SFU rate) over the measured step"}


def bench_c1(torch, R, stream, peaks, hbm_gbs, steps):
    """10K Gaussians, 128x128, plain single-view fwd+bwd (tile 16), L1 to a seeded target."""
    from paper_2501_14534_gb300 import synth
    w = synth.workload(1)
    g = R.Gaussians.from_numpy(w["scene"])
    cam = w["cams"][0]
    tgt = torch.from_numpy(w["targets"][0]).cuda()
    rast = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    loss = torch.zeros(1, device="cuda")
    dimg = torch.empty_like(tgt)
    grads = rast.alloc_grads(g)
    stats = rast.alloc_stats(g.n)
    count = 3 * cam.width * cam.height

    def view():
        outs = rast.forward(g, [cam])
        rast.l1_loss(outs[0]["image"], tgt, 1.0 / count, loss, dimg)
        rast.backward(g, [cam], outs, [dimg], grads, stats)

    with torch.cuda.stream(stream):
        for _ in range(5):
            view()
    stream.synchronize()
    n_t = max(20, steps)
    total, per = timed(torch, view, n_t, stream)
    # the same view through the batched step (one launch of each stage, no host sync)
    brast = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    brast.plan(g, [cam])
    with torch.cuda.stream(stream):
        for _ in range(3):
            brast.train_step_batched(g, [cam], [tgt], grads, None, loss, graph=True)
    stream.synchronize()
    btotal, bper = timed(torch, lambda: brast.train_step_batched(g, [cam], [tgt], grads, None, loss, graph=True),
                         n_t, stream)
    Pe, Pc = pair_counts(R, g, [cam], 16, 1, w["eps_mask"], w["eps_sh"])
    K = brast.plan(g, [cam])
    fl = step_floor_ms(g.n, 1, K, 64, count // 3, Pe, Pc, peaks, hbm_gbs)
    d = dist(per)
    return {"workload": w["name"], "metric": "plain fwd+bwd views/s", "value": 1000.0 * n_t / total,
            "unit": "views/s", "ms_per_step": d, "batched_step_views_per_s": 1000.0 * n_t / btotal,
            "batched_ms_per_step": dist(bper), "keys": K, "pairs": {"evaluated": Pe, "contributing": Pc},
            "roofline": _floor_record(fl, d["median"])}


def bench_c3(torch, R, stream, peaks, hbm_gbs, steps, autotune=True):
    """500K Gaussians, 16 mixed-resolution views (4 x 320x208, 6 x 640x416, 6 x 1280x832) in
    one batched step (persistent fused launch, CUDA graph), tile and pixels per thread tuned."""
    from paper_2501_14534_gb300 import synth
    w = synth.workload(3)
    cams = w["cams"]
    V = len(cams)
    g = R.Gaussians.from_numpy(w["scene"])
    tg = [torch.from_numpy(t).cuda() for t in w["targets"]]
    rast = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    tuned = rast.autotune(g, cams, tg) if autotune else None
    K = rast.plan(g, cams, headroom=1.15)
    grads = rast.alloc_grads(g)
    stats = rast.alloc_stats(g.n)
    loss = torch.zeros(1, device="cuda")

    def step():
        rast.train_step_batched(g, cams, tg, grads, stats, loss, graph=True)

    with torch.cuda.stream(stream):
        for _ in range(3):
            step()
    stream.synchronize()
    rast.poll()
    total, per = timed(torch, step, steps, stream)
    rast.poll()
    cfg = rast.config
    pixels = sum(c.width * c.height for c in cams)
    Pe, Pc = pair_counts(R, g, cams, cfg.tile, cfg.ppt, w["eps_mask"], w["eps_sh"])
    tiles = rast.num_tiles(cams)
    fl = step_floor_ms(g.n, V, K, tiles, pixels, Pe, Pc, peaks, hbm_gbs)
    d = dist(per)
    ms = total / steps
    return {"workload": w["name"], "metric": "fwd+bwd views/s (batched step)", "value": V * 1000.0 / ms,
            "unit": "views/s", "pixels_per_s": pixels * 1000.0 / ms, "ms_per_step": d,
            "tile": cfg.tile, "ppt": cfg.ppt, "autotuned": tuned is not None, "keys": K,
            "pairs": {"evaluated": Pe, "contributing": Pc}, "roofline": _floor_record(fl, d["median"])}


def bench_c4(torch, R, stream, peaks, hbm_gbs):
    """300K Gaussians with a per-Gaussian SH degree, 100 hemisphere poses at 1920x1080,
    forward only, one pose after another: FPS = 100 / total. The batched render
    (tgs_render_batched: no host synchronisation, key capacity planned once for the largest
    pose) is the value; the plain path (one key-count read per view) is reported beside it."""
    from paper_2501_14534_gb300 import synth
    w = synth.workload(4)
    cams = w["cams"]
    g = R.Gaussians.from_numpy(w["scene"])
    rast = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    outs = rast._alloc_views(cams[:1], g.n, want_state=False)
    camarr = [R.cameras_array([c]) for c in cams]
    k_max = max(rast.plan(g, [c]) for c in cams)
    rast.set(key_capacity=int(k_max * 1.15) + 1)

    def render(i):
        rast.render_batched(g, None, outs=outs, cams_struct=camarr[i])

    def render_plain(i):
        rast.forward(g, [cams[i]], want_state=False, outs=outs)

    with torch.cuda.stream(stream):
        for i in range(5):
            render(i)
            render_plain(i)
    stream.synchronize()
    rast.poll()
    it = iter(range(len(cams)))
    total, per = timed(torch, lambda: render(next(it)), len(cams), stream)
    rast.poll()
    it = iter(range(len(cams)))
    total_plain, _ = timed(torch, lambda: render_plain(next(it)), len(cams), stream)
    # throughput: 10 poses per call (10 calls for the 100 poses), capacity planned per group
    grp = 10
    groups = [cams[i:i + grp] for i in range(0, len(cams), grp)]
    brast = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    kg = max(brast.plan(g, gr) for gr in groups)
    brast.set(key_capacity=int(kg * 1.15) + 1)
    gouts = brast._alloc_views(groups[0], g.n, want_state=False)
    garr = [R.cameras_array(gr) for gr in groups]
    with torch.cuda.stream(stream):
        brast.render_batched(g, None, outs=gouts, cams_struct=garr[0])
    stream.synchronize()
    it = iter(range(len(groups)))
    total_grp, _ = timed(torch, lambda: brast.render_batched(g, None, outs=gouts, cams_struct=garr[next(it)]),
                         len(groups), stream)
    brast.poll()
    del brast, gouts
    # algorithmic work: SH coefficients read only up to each Gaussian's degree
    deg = w["scene"]["sh_degree"].astype(np.int64)
    param_bytes = float(np.mean(4 * (3 + 3 + 4 + 1 + 3) + 12 * ((deg + 1) ** 2 - 1)))
    Pe = Pc = K = 0
    counter = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    for c in cams[:10]:   # pair and key counts of 10 poses, scaled to the 100
        o = counter.forward(g, [c], want_examined=True, want_counts=True)[0]
        Pe += int(o["n_eval"].sum().item())
        Pc += int(o["n_contrib"].sum().item())
        sp, rd = counter.preprocess(g, [c])
        K += counter.bin(sp, rd, g.n, [c], want_keys=False)[3]
    f = len(cams) / 10
    fl = {k: v * f for k, v in step_floor_ms(g.n, 10, K, 10 * 8160, 10 * 1920 * 1080, Pe, Pc, peaks, hbm_gbs,
                                              backward=False, gbytes_param=10 * param_bytes).items()}
    # the 10-view floor counts the parameter read once per view, as a view-by-view render does
    algo_bytes = f * ((param_bytes + 48) * g.n * 10 + K * (12 + 24 * key_passes(8160) + 8 + 40)
                      + 12 * 1920 * 1080 * 10)
    d = dist(per)
    return {"workload": w["name"], "metric": "render FPS (forward only, batched render pose by pose)",
            "value": 1000.0 * len(cams) / total, "unit": "FPS", "ms_per_frame": d,
            "plain_path_fps": 1000.0 * len(cams) / total_plain, "key_capacity": int(k_max * 1.15) + 1,
            "fps_10_poses_per_call": 1000.0 * len(cams) / total_grp,
            "achieved_GBps": algo_bytes / (total * 1e-3) / 1e9,
            "keys_per_frame": K / 10, "pairs_per_frame": {"evaluated": Pe / 10, "contributing": Pc / 10},
            "roofline": _floor_record(fl, total)}


def bench_c5(torch, R, stream, peaks, hbm_gbs, steps):
    """3M Gaussians (256 blobs), 8 views of 1600x1064: the batched step, and the per-view
    checkpointed autograd path (forward of the 8 views keeping only T_final and last per view,
    then the backward re-binning each view); views/s and peak device memory."""
    from paper_2501_14534_gb300 import synth
    w = synth.workload(5)
    cams = w["cams"]
    V = len(cams)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    g = R.Gaussians.from_numpy(w["scene"])
    tg = [torch.from_numpy(t).cuda() for t in w["targets"]]
    rast = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    for k in R.PARAM_KEYS:
        t = getattr(g, k)
        if t is not None:
            t.requires_grad_(True)
    n_t = max(3, min(steps, 10))

    def ckpt_step():
        imgs = R.rasterize(rast, g, cams)
        loss = sum((im - t).abs().mean() for im, t in zip(imgs, tg)) / V
        loss.backward()

    with torch.cuda.stream(stream):
        for _ in range(3):   # warm-up: the allocator's blocks for the views' tensors settle
            ckpt_step()
    stream.synchronize()
    total, per = timed(torch, ckpt_step, n_t, stream)
    peak_ckpt = torch.cuda.max_memory_allocated() + rast.arena_bytes()
    for k in R.PARAM_KEYS:
        t = getattr(g, k)
        if t is not None:
            t.grad = None
            t.requires_grad_(False)
    # the batched step on the same scene and views
    brast = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    brast.autotune(g, cams, tg)
    K = brast.plan(g, cams, headroom=1.15)
    grads = brast.alloc_grads(g)
    loss = torch.zeros(1, device="cuda")

    def bstep():
        brast.train_step_batched(g, cams, tg, grads, None, loss, graph=True)

    with torch.cuda.stream(stream):
        for _ in range(3):
            bstep()
    stream.synchronize()
    brast.poll()
    btotal, bper = timed(torch, bstep, n_t, stream)
    cfg = brast.config
    pixels = sum(c.width * c.height for c in cams)
    Pe, Pc = pair_counts(R, g, cams, cfg.tile, cfg.ppt, w["eps_mask"], w["eps_sh"])
    fl = step_floor_ms(g.n, V, K, brast.num_tiles(cams), pixels, Pe, Pc, peaks, hbm_gbs)
    d = dist(per)
    bd = dist(bper)
    return {"workload": w["name"], "metric": "fwd+bwd views/s (per-view checkpointed autograd)",
            "value": V * 1000.0 * n_t / total, "unit": "views/s", "ms_per_step": d,
            "peak_device_bytes_checkpointed": int(peak_ckpt),
            "batched_step_views_per_s": V * 1000.0 * n_t / btotal, "batched_ms_per_step": bd,
            "batched_tile": cfg.tile, "batched_ppt": cfg.ppt, "keys": K,
            "peak_device_bytes": int(torch.cuda.max_memory_allocated() + rast.arena_bytes() + brast.arena_bytes()),
            "pairs": {"evaluated": Pe, "contributing": Pc},
            "roofline": _floor_record(fl, bd["median"])}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_14534_gb300 import build as tgs_build
    tgs_build.build()
    from paper_2501_14534_gb300 import rasterizer as R

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        peaks = R.Rasterizer.measure_peaks()
    hbm_gbs, peak_kind = load_peaks()

    w = workload(args.n, args.views)
    cams = w["cams"]
    V = len(cams)
    g = R.Gaussians.from_numpy(w["scene"])
    targets = [torch.from_numpy(t).cuda() for t in w["targets"]]
    rast = R.Rasterizer(tile=args.tile, ppt=args.ppt, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    tuned = None
    if not args.no_autotune:
        t0 = time.time()
        tuned = rast.autotune(g, cams, targets)
        print(f"[bench] autotune {tuned} in {time.time() - t0:.1f} s", file=sys.stderr)
    K_keys = rast.plan(g, cams, headroom=1.15)
    grads = rast.alloc_grads(g)
    stats = rast.alloc_stats(g.n)
    loss = torch.zeros(1, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def step():
        rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True)

    # warm-up; the timed graph carries no profiling events
    rast.set_profiling(False)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    rast.poll()
    kernels = rast.kernels_per_step()

    # ---- timed region: K batched steps back to back (inputs in HBM, larger than L2) ----
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        total_ms, per_step = timed(torch, step, args.steps, stream)
    barrier()
    from paper_2501_14534_gb300 import dist as tgs_dist
    ms_total = tgs_dist.reduce_max(total_ms, device="cuda")   # max over ranks
    rast.poll()
    ms_step = ms_total / args.steps
    value = V * world / (ms_step / 1000.0)

    # ---- per-stage times: a few more steps with events between the stages (in the graph) ----
    rast.set_profiling(True)
    stage_sum = {}
    n_prof = 3
    with torch.cuda.stream(stream):
        step()   # captures the profiled graph
        stream.synchronize()
        for _ in range(n_prof):
            step()
            for k, v in rast.stage_times().items():   # synchronises on the step's last event
                stage_sum[k] = stage_sum.get(k, 0.0) + v
    stream.synchronize()
    rast.set_profiling(False)
    stage_ms = {k: v / n_prof for k, v in stage_sum.items()}

    if args.step_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "views/s", "partial": True,
                              "ms_per_step": ms_step, "step_ms": dist(per_step), "stage_ms": stage_ms,
                              "kernels_per_step": kernels}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- A/B: the same step with separate forward, loss and backward kernels ----
    unfused = None
    try:
        with torch.cuda.stream(stream):
            for _ in range(2):
                rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True, fused=False)
        stream.synchronize()
        t, _ = timed(torch, lambda: rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True,
                                                             fused=False), 3, stream)
        unfused = V * world / (t / 3 / 1000.0)
    except Exception as e:  # reported, not fatal
        print(f"[bench] unfused A/B failed: {e}", file=sys.stderr)

    # ---- the step with the L1 + D-SSIM loss of Eq. loss3dgs (separate launches) ----
    dssim = None
    try:
        with torch.cuda.stream(stream):
            for _ in range(2):
                rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True, dssim=True)
        stream.synchronize()
        t, _ = timed(torch, lambda: rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True,
                                                             dssim=True), 3, stream)
        dssim = {"views_per_s": V * world / (t / 3 / 1000.0)}
        rast.set_profiling(True)
        with torch.cuda.stream(stream):
            for _ in range(2):   # the first captures the profiled graph
                rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True, dssim=True)
            dssim["stage_ms"] = rast.stage_times()
        rast.set_profiling(False)
        ms = dssim["stage_ms"].get("l1_dssim_loss")
        if ms:
            elems = 3 * sum(c.width * c.height for c in cams)
            # algorithmic bytes: read image and target, write dL/dimage (4 B each per element)
            dssim["loss_kernels"] = {"elements": elems, "ms": ms, "algorithmic_GBps": 12 * elems / ms / 1e6}
    except Exception as e:  # reported, not fatal
        rast.set_profiling(False)
        print(f"[bench] D-SSIM step failed: {e}", file=sys.stderr)

    # ---- e2e: one C-ABI call per step with the inputs in pinned host memory (the library
    # copies them in on its upload stream and copies the loss back) ----
    hostg = R.Gaussians(**{k: t.detach().cpu().pin_memory() for k, t in g.params().items()},
                        sh_degree_max=g.sh_degree_max)
    host_t = [t.cpu().pin_memory() for t in targets]
    h2d = sum(t.numel() * t.element_size() for t in hostg.params().values()) + \
        sum(t.numel() * t.element_size() for t in host_t)
    loss_host = torch.zeros(1).pin_memory()
    camarr = R.cameras_array(cams)

    def e2e_step():
        rast.train_step_batched_host(hostg, cams, host_t, grads, stats, loss_host, graph=True, cams_struct=camarr)

    with torch.cuda.stream(stream):
        for _ in range(4):   # every buffer set filled and its graph captured
            e2e_step()
    stream.synchronize()
    n_e2e = max(5, args.steps)   # as many steps as the device-resident timing
    barrier()
    torch.cuda.synchronize()
    e2e_total, e2e_per = timed(torch, e2e_step, n_e2e, stream)
    torch.cuda.synchronize()   # the last loss copy has landed in loss_host
    e2e_ms = e2e_total / n_e2e
    e2e_value = V * world / (e2e_ms / 1000.0)

    # ---- the plain single-view path and forward-only FPS on the same views ----
    def plain_rate(tile, ppt, backward=True, gg=None):
        gg = gg or g
        plain = R.Rasterizer(tile=tile, ppt=ppt, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
        pl_loss = torch.zeros(1, device="cuda")
        dimg = [torch.empty_like(t) for t in targets]
        pgrads = plain.alloc_grads(gg) if backward else None
        pstats = plain.alloc_stats(gg.n) if backward else None

        def one(v):
            outs = plain.forward(gg, [cams[v]])
            if backward:
                plain.l1_loss(outs[0]["image"], targets[v], 1.0 / (3 * W * H * V), pl_loss, dimg[v])
                plain.backward(gg, [cams[v]], outs, [dimg[v]], pgrads, pstats, accumulate=v > 0)

        with torch.cuda.stream(stream):
            for v in range(min(V, 3)):
                one(v)
        stream.synchronize()
        it = iter(range(V))
        t, _ = timed(torch, lambda: one(next(it)), V, stream)
        return V / (t / 1000.0)

    cfg0 = rast.config
    plain_vps = plain_rate(16, 1)
    plain_by_cfg = {}
    for tl, pp in [(8, 1), (8, 2), (16, 2), (16, 4), (32, 2), (32, 4)]:
        plain_by_cfg[f"{tl}x{pp}"] = plain_rate(tl, pp)
    plain_by_cfg["16x1"] = plain_vps
    best_cfg = max(plain_by_cfg, key=plain_by_cfg.get)
    plain_best = plain_by_cfg[best_cfg]
    render_fps = plain_rate(16, 1, backward=False)
    # forward only through the batched render: the 16 views per call, graph replayed
    rrast = R.Rasterizer(tile=cfg0.tile, ppt=cfg0.ppt, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    rrast.plan(g, cams, headroom=1.15)
    routs = rrast._alloc_views(cams, g.n, want_state=False)
    with torch.cuda.stream(stream):
        for _ in range(3):
            rrast.render_batched(g, cams, outs=routs, graph=True)
    stream.synchronize()
    t, _ = timed(torch, lambda: rrast.render_batched(g, cams, outs=routs, graph=True), 10, stream)
    rrast.poll()
    render_fps_batched = 10 * V / (t / 1000.0)
    del rrast, routs
    # the same render from FP16 parameter storage (the paper's post-processing)
    gh = R.Rasterizer.to_half(g)
    render_fps_fp16 = plain_rate(16, 1, backward=False, gg=gh)
    del gh

    # ---- a significance pruning round on the same scene (Eq. significance-score): ray hits
    # over the views, score, selection of the lowest 60 %, compaction of every parameter array
    pruning = None
    if not args.no_pruning_round:
        try:
            prast = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])

            def prune_round():
                # each stage bracketed by events with the device idle before it, so that a gap on
                # the host (a first launch, an allocation) is not counted as device time
                ms = []
                out = []
                stages = [lambda: prast.count_hits(g, cams), lambda: prast.significance(g, out[0], 0.9),
                          lambda: prast.prune_select(out[1], 0.6), lambda: prast.compact(g, out[2], masked=True)[0]]
                for f in stages:
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    out.append(f())
                    e1.record()
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                return ms, out[3]

            prune_round()   # first launches and buffer growth, untimed
            ms, kept = prune_round()
            prast.poll()
            # a binning of the pruned scene in the same context (its scratch reused)
            sp, rd = prast.preprocess(kept, cams[:1])
            K_pruned = prast.bin(sp, rd, kept.n, cams[:1], want_keys=False)[3]
            prast.poll()
            # kept rows read and written, index map written, removal flag and mask logit read
            moved = 2 * kept.n * 252 + 4 * kept.n + 5 * g.n
            pruning = {"gaussians": g.n, "kept": kept.n, "count_hits_ms": ms[0], "significance_ms": ms[1],
                       "prune_select_ms": ms[2], "compact_ms": ms[3],
                       "compact_GBps": moved / ms[3] / 1e6, "keys_view0_after": K_pruned}
            del kept
        except Exception as e:  # reported, not fatal
            print(f"[bench] pruning round failed: {e}", file=sys.stderr)

    # ---- roofline of the dominant kernel: algorithmic work from exact pair counts at the
    # batched step's tile size, over the stage's average CUDA-event time ----
    cfg = rast.config
    P_eval, P_contrib = pair_counts(R, g, cams, cfg.tile, cfg.ppt, w["eps_mask"], w["eps_sh"])
    n = g.n
    bytes_pre = n * 252 + V * n * (48 + 4 + 4 + 4 + 48)
    bytes_pbwd = n * (252 + 252 + 12 * 2) + V * n * (48 + 4)
    ops_fwd = P_eval * OPS_EVAL + P_contrib * OPS_BLEND
    ops_bwd = P_contrib * OPS_BWD
    fp32_peak = peaks["fp32_fma_per_s"] / 1e12
    work = {
        "fused_blend": ("alu", (ops_fwd + ops_bwd) / 1e12, fp32_peak, "Tops/s"),
        "preprocess": ("hbm", bytes_pre / 1e9, hbm_gbs, "GB/s"),
        "preprocess_backward": ("hbm", bytes_pbwd / 1e9, hbm_gbs, "GB/s"),
        "blend_forward": ("alu", ops_fwd / 1e12, fp32_peak, "Tops/s"),
        "blend_backward": ("alu", ops_bwd / 1e12, fp32_peak, "Tops/s"),
    }
    dom = max((k for k in stage_ms if k in work), key=lambda k: stage_ms[k])
    bound, units, peak, unit = work[dom]
    achieved = units / (stage_ms[dom] / 1000.0)
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak,
                "traffic": fused_traffic(cfg, n, V) if dom == "fused_blend" else None,
                "peak_source": (f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if bound == "hbm" else
                                "measured: scalar fma.rn.f32 issue rate of tgs_measure_peaks")}
    if dom == "fused_blend":
        sfu_ops = SFU_PER_CONTRIB * P_contrib
        roofline["sfu"] = {"achieved": sfu_ops / (stage_ms[dom] / 1000.0) / 1e12,
                           "peak": peaks["ex2_per_s"] / 1e12, "unit": "T ops/s",
                           "frac": sfu_ops / (stage_ms[dom] / 1000.0) / peaks["ex2_per_s"]}
    floor = step_floor_ms(n, V, K_keys, rast.num_tiles(cams), V * W * H, P_eval, P_contrib, peaks, hbm_gbs)
    step_roofline = _floor_record(floor, dist(per_step)["median"])

    # ---- the other workloads ----
    subs = None
    if not args.no_workloads and rank == 0:
        subs = {}
        for key, fn in [("plain_10k_128x128", lambda: bench_c1(torch, R, stream, peaks, hbm_gbs, args.steps)),
                        ("batched_500k_16_mixed_views", lambda: bench_c3(torch, R, stream, peaks, hbm_gbs,
                                                                         args.steps, not args.no_autotune)),
                        ("render_300k_1920x1080_100_poses", lambda: bench_c4(torch, R, stream, peaks, hbm_gbs)),
                        ("large_3m_8x1600x1064", lambda: bench_c5(torch, R, stream, peaks, hbm_gbs, args.steps))]:
            try:
                t0 = time.time()
                subs[key] = fn()
                print(f"[bench] {key}: {time.time() - t0:.1f} s", file=sys.stderr)
            except Exception as e:  # reported, not fatal
                subs[key] = {"error": str(e)}
                print(f"[bench] {key} failed: {e}", file=sys.stderr)
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        wv = dict(w, cams=w["cams"][:1], targets=w["targets"][:1])
        v, cores, desc, _ = cpu_baseline(wv)
        cpu = {"value": v, "unit": "views/s", "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "step_ms": dist(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w["name"], "global_batch": V * world, "views_per_gpu": V,
                       "width": W, "height": H, "gaussians": n, "keys": K_keys,
                       "tile": cfg.tile, "ppt": cfg.ppt, "autotuned": tuned is not None,
                       "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (252 MB params)"},
            "e2e": {"value": e2e_value, "unit": "views/s", "steps": n_e2e, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": 4, "ms_per_step": e2e_ms, "step_ms": dist(e2e_per),
                    "api": "tgs_train_step_batched_host (pinned host inputs, copies on the library's upload "
                           "stream into three buffer sets, overlapping the previous steps)"},
            "plain_views_per_s": plain_vps, "plain_best": {"config": best_cfg, "views_per_s": plain_best},
            "plain_by_config": plain_by_cfg,
            "render_fps": render_fps, "render_fps_fp16_params": render_fps_fp16,
            "render_fps_batched": render_fps_batched,
            "pruning_round": pruning,
            "unfused_views_per_s": unfused, "l1_dssim_step": dssim,
            "speedup_vs_plain": value / world / plain_vps,
            "speedup_vs_plain_best": value / world / plain_best,
            "stage_ms": stage_ms,
            "pairs": {"evaluated": P_eval, "contributing": P_contrib},
            "peaks": {k: peaks[k] for k in ("fp32_fma_per_s", "fp32x2_fma_per_s", "ex2_per_s", "rcp_per_s")},
            "roofline": roofline, "step_roofline": step_roofline,
            "workloads": subs,
            "cpu_baseline": cpu, "clocks": clk.summary(),
            "gpu_launches": kernels * args.steps,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
