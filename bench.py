#!/usr/bin/env python
"""Benchmark of the rasterizer hot path: one step = one batched training step (preprocess,
binning, forward blend, L1 loss, backward blend, preprocess backward) over 16 views of
1280x832 of a 1M-Gaussian masked scene (64 blobs + 10% shell, SH degree 3, volume and
SH-band masks at eps = 0.5).

Prints one JSON line. value = views per second of the batched step with inputs resident in
HBM; e2e = the same through the C ABI with the Gaussian parameters and target images copied
from pinned host memory every step and the loss read back. Also reports the plain
single-view path (views/s) and forward-only render FPS for comparison, the roofline of the
dominant kernel, and the FP64 CPU oracle timed on the host cores on a bounded sample.

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
# float32 lanes: 152 SMs x 128 lanes x 2.07 GHz max SM clock
ALU_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12
# DRAM bytes (read + write) of one fused-blend launch on the default workload at tile 32,
# 2 px/thread, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum; the command
# is in profiles/k_fused_l1_300k_8x1280x832_tile32_ppt2.md). Reported only while the kernel's
# sources and the code that launches it are the ones measured (their sha256 below), else null.
FUSED_TRAFFIC = {"bytes": 718457344 + 96854016, "tile": 32, "ppt": 2,
                 "sources": ("fused.cu", "blend_common.cuh", "tgs_internal.cuh", "api.cu"),
                 "sha256": "cc74fd57e338fde486bf9de8879cbab239d673303cfc183c29aeb7391ca3219f"}


def fused_traffic(cfg, n, views):
    import hashlib
    t = FUSED_TRAFFIC
    if (cfg.tile, cfg.ppt, n, views) != (t["tile"], t["ppt"], N_GAUSS, N_VIEWS):
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
    p.add_argument("--tile", type=int, default=16)
    p.add_argument("--ppt", type=int, default=1)
    p.add_argument("--pruning-round", action="store_true",
                   help="also time a significance pruning round (hits, score, selection, compaction)")
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
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_14534_gb300 import build as tgs_build
    tgs_build.build()
    from paper_2501_14534_gb300 import rasterizer as R

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
    stream = torch.cuda.Stream()

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
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
        stream.synchronize()
    barrier()
    from paper_2501_14534_gb300 import dist as tgs_dist
    ms_total = tgs_dist.reduce_max(e0.elapsed_time(e1), device="cuda")   # max over ranks
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
                              "ms_per_step": ms_step, "stage_ms": stage_ms,
                              "kernels_per_step": kernels}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- A/B: the same step with separate forward, loss and backward kernels ----
    rast.set_profiling(False)
    unfused = None
    try:
        with torch.cuda.stream(stream):
            for _ in range(2):
                rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True, fused=False)
            u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            u0.record(stream)
            for _ in range(3):
                rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True, fused=False)
            u1.record(stream)
        stream.synchronize()
        unfused = V * world / (u0.elapsed_time(u1) / 3 / 1000.0)
    except Exception as e:  # reported, not fatal
        print(f"[bench] unfused A/B failed: {e}", file=sys.stderr)

    # ---- the step with the L1 + D-SSIM loss of Eq. loss3dgs (separate launches) ----
    dssim = None
    try:
        with torch.cuda.stream(stream):
            for _ in range(2):
                rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True, dssim=True)
            d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            d0.record(stream)
            for _ in range(3):
                rast.train_step_batched(g, cams, targets, grads, stats, loss, graph=True, dssim=True)
            d1.record(stream)
        stream.synchronize()
        dssim = {"views_per_s": V * world / (d0.elapsed_time(d1) / 3 / 1000.0)}
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

    # ---- e2e: inputs from pinned host memory each step, loss read back ----
    host = {k: t.detach().cpu().pin_memory() for k, t in g.params().items()}
    host_t = [t.cpu().pin_memory() for t in targets]
    h2d = sum(t.numel() * t.element_size() for t in host.values()) + \
        sum(t.numel() * t.element_size() for t in host_t)
    loss_host = torch.zeros(1).pin_memory()
    rast.set_profiling(False)
    with torch.cuda.stream(stream):
        step()
    stream.synchronize()
    n_e2e = max(2, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n_e2e):
            for k, t in g.params().items():
                t.copy_(host[k], non_blocking=True)
            for t, h in zip(targets, host_t):
                t.copy_(h, non_blocking=True)
            step()
            loss_host.copy_(loss, non_blocking=True)
        a1.record(stream)
    stream.synchronize()
    e2e_ms = a0.elapsed_time(a1) / n_e2e
    e2e_value = V * world / (e2e_ms / 1000.0)

    # ---- the plain single-view path and forward-only FPS on the same views ----
    plain = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    pl_loss = torch.zeros(1, device="cuda")
    dimg = [torch.empty_like(t) for t in targets]
    pgrads = plain.alloc_grads(g)
    pstats = plain.alloc_stats(g.n)

    def plain_view(v, backward=True):
        outs = plain.forward(g, [cams[v]])
        if backward:
            plain.l1_loss(outs[0]["image"], targets[v], 1.0 / (3 * W * H * V), pl_loss, dimg[v])
            plain.backward(g, [cams[v]], outs, [dimg[v]], pgrads, pstats, accumulate=v > 0)
        return outs

    for v in range(min(V, 3)):
        plain_view(v)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for v in range(V):
        plain_view(v)
    p1.record()
    torch.cuda.synchronize()
    plain_vps = V / (p0.elapsed_time(p1) / 1000.0)
    p0.record()
    for v in range(V):
        plain_view(v, backward=False)
    p1.record()
    torch.cuda.synchronize()
    render_fps = V / (p0.elapsed_time(p1) / 1000.0)
    # the same render from FP16 parameter storage (the paper's post-processing)
    gh = R.Rasterizer.to_half(g)
    for v in range(min(V, 3)):
        plain.forward(gh, [cams[v]])
    p0.record()
    for v in range(V):
        plain.forward(gh, [cams[v]])
    p1.record()
    torch.cuda.synchronize()
    render_fps_fp16 = V / (p0.elapsed_time(p1) / 1000.0)
    del gh

    # ---- a significance pruning round on the same scene (Eq. significance-score): ray hits
    # over the views, score, selection of the lowest 60 %, compaction of every parameter array
    pruning = None
    if args.pruning_round:
        try:
            def prune_round():
                # each stage bracketed by events with the device idle before it, so that a gap on
                # the host (a first launch, an allocation) is not counted as device time
                ms = []
                out = []
                stages = [lambda: plain.count_hits(g, cams), lambda: plain.significance(g, out[0], 0.9),
                          lambda: plain.prune_select(out[1], 0.6), lambda: plain.compact(g, out[2], masked=True)[0]]
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
            # kept rows read and written, index map written, removal flag and mask logit read
            moved = 2 * kept.n * 252 + 4 * kept.n + 5 * g.n
            pruning = {"gaussians": g.n, "kept": kept.n, "count_hits_ms": ms[0], "significance_ms": ms[1],
                       "prune_select_ms": ms[2], "compact_ms": ms[3],
                       "compact_GBps": moved / ms[3] / 1e6}
            del kept
        except Exception as e:  # reported, not fatal
            print(f"[bench] pruning round failed: {e}", file=sys.stderr)

    # algorithmic work of the blend stages: pairs examined per pixel (forward) and pairs up to
    # the last contributor (backward), from a forward with per-pixel counters at the tile size
    # of the batched step
    cfg = rast.config
    counter = R.Rasterizer(tile=cfg.tile, ppt=cfg.ppt, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    P_exam = P_eval = P_contrib = 0
    for v in range(V):
        o = counter.forward(g, [cams[v]], want_examined=True, want_counts=True)[0]
        P_exam += int(o["n_examined"].sum().item())
        P_eval += int(o["n_eval"].sum().item())
        P_contrib += int(o["n_contrib"].sum().item())
    hbm_gbs, peak_kind = load_peaks()
    n = g.n
    bytes_pre = n * 252 + V * n * (48 + 4 + 4 + 4 + 48)
    bytes_pbwd = n * (252 + 252 + 12 * 2) + V * n * (48 + 4)
    ops_fwd = P_eval * OPS_EVAL + P_contrib * OPS_BLEND
    ops_bwd = P_contrib * OPS_BWD
    work = {
        "fused_blend": ("alu", (ops_fwd + ops_bwd) / 1e12, ALU_PEAK_TOPS, "Tops/s"),
        "preprocess": ("hbm", bytes_pre / 1e9, hbm_gbs, "GB/s"),
        "preprocess_backward": ("hbm", bytes_pbwd / 1e9, hbm_gbs, "GB/s"),
        "blend_forward": ("alu", ops_fwd / 1e12, ALU_PEAK_TOPS, "Tops/s"),
        "blend_backward": ("alu", ops_bwd / 1e12, ALU_PEAK_TOPS, "Tops/s"),
    }
    dom = max((k for k in stage_ms if k in work), key=lambda k: stage_ms[k])
    bound, units, peak, unit = work[dom]
    achieved = units / (stage_ms[dom] / 1000.0)
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak,
                "traffic": fused_traffic(cfg, n, V) if dom == "fused_blend" else None,
                "peak_source": (f"{peak_kind} hbm_gbs" if bound == "hbm" else
                                "152 SMs x 128 FP32 lanes x 2.07 GHz")}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        wv = dict(w, cams=w["cams"][:1], targets=w["targets"][:1])
        v, cores, desc, _ = cpu_baseline(wv)
        cpu = {"value": v, "unit": "views/s", "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w["name"], "global_batch": V * world, "views_per_gpu": V,
                       "width": W, "height": H, "gaussians": n, "keys": K_keys,
                       "tile": cfg.tile, "ppt": cfg.ppt, "autotuned": tuned is not None,
                       "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (252 MB params)"},
            "e2e": {"value": e2e_value, "unit": "views/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": 4, "ms_per_step": e2e_ms},
            "plain_views_per_s": plain_vps, "render_fps": render_fps, "render_fps_fp16_params": render_fps_fp16,
            "pruning_round": pruning,
            "unfused_views_per_s": unfused, "l1_dssim_step": dssim,
            "speedup_vs_plain": value / world / plain_vps,
            "stage_ms": stage_ms,
            "pairs": {"examined": P_exam, "evaluated": P_eval, "contributing": P_contrib},
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk.summary(),
            "gpu_launches": kernels * args.steps,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
