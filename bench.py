#!/usr/bin/env python3
"""Benchmark of the PackUV-GS render step (forward + backward) on GB300.

One step = one fitting iteration over every view of the workload: atlas
gather, projection + SH, binning + sort, forward compositing, L1 loss
gradient, backward compositing, texel-gradient scatter -- all views in one
sequence of launches, captured once in a CUDA graph and replayed.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on bounded samples of the same workload instead.
"""

from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "fwd+bwd rendered MPix/s on 1 GB300, batched vs per-view, % of HBM roofline"
UNIT = "MPix/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
FP32_LANES_PER_SM = 128


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

def _cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def gpu_local_affinity(dev_index):
    """Restrict this process to the CPUs local to the GPU (from sysfs);
    returns (previous affinity or None, a short description)."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev_index)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        local = _cpulist(open("/sys/bus/pci/devices/%s/local_cpulist" % bus).read()) & os.sched_getaffinity(0)
        if not local:
            return None, "unchanged (no local CPUs listed for %s)" % bus
        before = os.sched_getaffinity(0)
        os.sched_setaffinity(0, local)
        return before, "%d CPUs local to %s" % (len(local), bus)
    except Exception as ex:  # no sysfs entry or property: leave the affinity alone
        return None, "unchanged (%s)" % type(ex).__name__


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes of one step (the byte model of the method)
# ---------------------------------------------------------------------------

def algorithmic_bytes(plan, texel_bytes, dups, n_dyn):
    N, V, D, P = plan.N, plan.V, plan.D, plan.P
    G = plan.G
    return {
        "a1_atlas_gather": G * D * texel_bytes + G * D * 4,
        "a2_project_and_sh": G * D * 4 + plan.pairs * 48,
        "a3_bin_and_sort": dups * (12 + 24),
        "a4_rasterize_fwd_l1": dups * 40 + P * 20 + P * 24,   # + target read, dL/dimage write
        "a5_rasterize_bwd": dups * 40 + P * 20 + plan.pairs * 36,
        "a6_atlas_scatter_grad": G * D * 4 + plan.pairs * 36 + n_dyn * D * 4,
    }


# Sources of each rooflined kernel: the DRAM traffic measured by ncu is
# reported only while these still hash to the profiled version.
KERNEL_SOURCES = {
    "a4_rasterize_fwd_l1": ("k_raster_fwd", ["pk_raster_fwd.cu", "pk_raster.cuh", "pk_f32x2.cuh", "pk_common.cuh",
                                             "pk_tma.cuh"]),
    "a5_rasterize_bwd": ("k_raster_bwd", ["pk_raster_bwd.cu", "pk_raster.cuh", "pk_f32x2.cuh", "pk_common.cuh",
                                          "pk_tma.cuh"]),
}


def measured_traffic(stage, dups):
    """Bytes per launch = ncu bytes per entry (small case) x this launch's entries, or None."""
    import hashlib
    if stage not in KERNEL_SOURCES:
        return None, None
    kernel, files = KERNEL_SOURCES[stage]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2602_23040_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    digest = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "traffic_per_entry.md")
    if not os.path.exists(path):
        return None, None
    with open(path) as fh:
        for line in fh:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) == 3 and cells[0] == kernel:
                if cells[1] != digest:
                    return None, "kernel changed since its ncu capture"
                return float(cells[2]) * dups, "ncu C3 4-view capture, bytes per entry x entries"
    return None, None


def measured_fp32_per_eval(stage):
    """FP32 lane operations and issued thread instructions per (pixel, splat)
    evaluation of a compositing kernel, from the committed ncu counters
    (profiles/fp32_per_evaluation.md: FADD + FMUL + FFMA + 2 x (FADD2 + FMUL2
    + FFMA2) thread instructions, predicated on, over the launch's
    evaluations), while the kernel's sources still hash to the profiled
    version; else None."""
    import hashlib
    if stage not in KERNEL_SOURCES:
        return None
    kernel, files = KERNEL_SOURCES[stage]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2602_23040_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    digest = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "fp32_per_evaluation.md")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 5 and cells[0] == kernel and cells[1] == digest:
                return {"fp32_lane_ops": float(cells[2]), "thread_inst": float(cells[3]),
                        "issue_active_pct": float(cells[4]), "source": "ncu counters, 52-view rig cut to 4 views"}
    return None


def launches_per_step(plan):
    # gather 2, project 1, bin_and_sort (as the library counts it), fwd with the loss 2 (zeroing +
    # compositing), bwd 2 (zeroing + adjoint), scatter 1
    return 2 + 1 + int(plan.sizes.bin_kernels) + 5


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on bounded windows of the workload's views
# ---------------------------------------------------------------------------

def window_views(scene, n, size, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in rng.choice(len(scene.views), n, replace=False):
        v = scene.views[int(i)]
        w, h = min(size, v.width), min(size, v.height)
        x0, y0 = (v.width - w) // 2, (v.height - h) // 2
        out.append(synth.View(R=v.R, t=v.t, fx=v.fx, fy=v.fy, cx=v.cx - x0, cy=v.cy - y0, width=w, height=h,
                              frame=v.frame))
    return out


def oracle_step(orc, scene, views, soa, texel, dynflag, target_seed=0, keep=None):
    """One oracle fwd + L1 + bwd over `views`; returns pixels rendered.  With
    `keep` (a list), appends the step's image, transmittance, borderline
    bits, flip bounds, dL/dimage and texel gradient to it."""
    va = orc.views_array(views)
    N = len(texel)
    rec = orc.project(soa, N, scene.sh_degree, va)
    vals, ranges = orc.bin_sort(rec, va, 16)
    r = orc.render(rec, va, 16, vals, ranges)
    P = int(sum(v.width * v.height for v in views))
    tgt = np.random.default_rng(target_seed).uniform(0, 1, 3 * P)
    dimg = np.sign(r["img"] - tgt) / (3 * P)
    g2 = orc.render_bwd(rec, va, 16, vals, ranges, dimg)
    g = orc.scatter_grad(soa, N, scene.sh_degree, va, g2, dynflag if scene.dyn is not None else None)
    if keep is not None:
        keep.append(dict(img=r["img"], T=r["T"], border=r["border"], bound=r["bound"], dimg=dimg, grad=g, P=P))
    return P


def cpu_baseline(scene, budget_s=20.0, window=256):
    """The oracle timed on view windows of the workload; also returns the
    windows and the oracle's outputs on them (for the accuracy check)."""
    import oracle as orc
    soa, texel, dynflag = orc.gather(scene)
    t0 = time.perf_counter()
    pix, n = 0, 0
    views = window_views(scene, min(8, len(scene.views)), window)
    kept = []
    while n < len(views) and (time.perf_counter() - t0) < budget_s:
        pix += oracle_step(orc, scene, [views[n]], soa, texel, dynflag, n, keep=kept)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": pix / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} view windows of {window}x{window} px from {scene.name}, all {scene.n_live} "
                      f"Gaussians each, fwd + L1 + bwd in FP64, single thread",
            "seconds": dt}, views[:n], kept


GROUPS = {"position": (0, 3), "log_scale": (3, 6), "rotation": (6, 10), "opacity": (10, 11), "sh_dc": (11, 14),
          "sh_rest": (14, None)}
IMAGE_BORDER = 1 | 2 | 4 | 8 | 16   # the oracle's borderline bits of image decisions


def accuracy_on_windows(scene, views, kept, atlas, occ, dyn, dev):
    """The library on the CPU-baseline's view windows, all in one launch,
    against the oracle's outputs there: image error off the borderline
    pixels, the largest excess over a borderline pixel's flip bound (<= 0:
    every pixel within), the borderline fractions, and the relative error of
    each attribute group of the texel gradient for the oracle's own
    dL/dimage."""
    import torch
    import paper_2602_23040_gb300 as pk
    if not kept:
        return None
    r = pk.Renderer(pk.Plan.for_scene(scene, views=views, tile=32), dev)
    r.ensure_capacity(atlas, occ, dyn)
    F, D, Hh, W = scene.atlas.shape
    dimg = torch.from_numpy(np.concatenate([k["dimg"] for k in kept]).astype(np.float32)).to(dev)
    grad = torch.zeros(F * D * Hh * W, dtype=torch.float32, device=dev)
    r.backward(dimg, grad)
    torch.cuda.synchronize(dev)
    st = r.status()
    img = r.image.cpu().numpy().astype(np.float64)
    T = r.T.cpu().numpy().astype(np.float64)
    texel = r.texel[:r.plan.N].cpu().numpy().view(np.uint32)
    g = grad.view(F, D, Hh * W).cpu().numpy().astype(np.float64)
    g = np.concatenate([g[f][:, texel] for f in range(F)], axis=1)
    ref = sum(k["grad"] for k in kept)
    off, worst_off, excess, nb, nt = 0, 0.0, -1.0, 0, 0
    for k in kept:
        P = k["P"]
        b = (k["border"] & IMAGE_BORDER) != 0
        nb += int(b.sum())
        nt += int(((k["border"] & (IMAGE_BORDER & ~8)) != 0).sum())
        for c in range(3):
            e = np.abs(img[3 * off + c * P:3 * off + (c + 1) * P] - k["img"][c * P:(c + 1) * P])
            worst_off = max(worst_off, float(e[~b].max(initial=0.0)))
            excess = max(excess, float((e - k["bound"][:, 0]).max()))
        excess = max(excess, float((np.abs(T[off:off + P] - k["T"]) - k["bound"][:, 1]).max()))
        off += P
    rel = {}
    for name, (a, bnd) in GROUPS.items():
        den = np.linalg.norm(ref[a:bnd])
        if den > 0:
            rel[name] = float(np.linalg.norm(g[a:bnd] - ref[a:bnd]) / den)
    return {"image_max_abs_err_off_borderline": worst_off, "image_max_excess_over_flip_bound": excess,
            "image_tolerance": 1e-4,
            "borderline_frac": nb / off, "threshold_borderline_frac": nt / off, "pixels": off,
            "grad_rel_err": rel, "status_flags": int(st["flags"]),
            "sample": f"the CPU baseline's {len(kept)} view windows, one launch (32 px tiles); oracle FP64"}


def _oracle_worker(args):
    """One process of the all-core oracle baseline: its own copy of the
    scene, its own view windows; returns (pixels, compute seconds)."""
    config, n_views, window, seed = args
    import oracle as orc
    scene = synth.config_scene(config, n_views=n_views or None)
    soa, texel, dynflag = orc.gather(scene)
    views = window_views(scene, 1, window, seed=seed)
    t0 = time.perf_counter()
    pix = oracle_step(orc, scene, views, soa, texel, dynflag, seed)
    return pix, time.perf_counter() - t0


def cpu_baseline_all_cores(config, n_views, window=256):
    """The same oracle, one process per host core (spawned), each rendering
    one window: pixels of all processes over the slowest process's time."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(config, n_views, window, 100 + i) for i in range(cores)])
    pix = sum(r[0] for r in res)
    slow = max(r[1] for r in res)
    return {"value": pix / slow / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes x one {window}x{window} px view window, fwd + L1 + bwd in FP64",
            "seconds": slow}


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle, on bounded samples of the same workload."""
    if rank != 0:
        return 0
    import oracle as orc
    scene = synth.config_scene(args.config)
    soa, texel, dynflag = orc.gather(scene)
    views = window_views(scene, len(scene.views), args.ref_window, seed=1)
    times, pix = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        p = oracle_step(orc, scene, [views[i % len(views)]], soa, texel, dynflag, i)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            pix += p
    total = sum(times)
    value = pix / total / 1e6
    cores = 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": scene.name, "sample": f"one {args.ref_window}x{args.ref_window} px window "
                                                         f"of one view per step, all {scene.n_live} Gaussians"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.ref_window}x{args.ref_window} px window per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def next_rows(plan, r, scene, atlas, occ, target, stream, dev, hbm):
    """The rows after the render step, timed at the same workload: motion
    masks and the dynamic mask (Alg. 1), the LPO proxy, Max-K UV pruning and
    the L1 + D-SSIM objective.  Each: median of 5 eager calls (CUDA events on
    the launching stream, L2 flushed between calls) and its HBM roofline."""
    import torch
    import paper_2602_23040_gb300 as pk
    F, D, Hh, W = scene.atlas.shape
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, reps=5):
        with torch.cuda.stream(stream):
            for _ in range(2):
                fn()
            ts = []
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    def row(ms, nbytes, unit_count, unit):
        return {"ms": ms, "algorithmic_bytes": int(nbytes), "achieved_gbs": nbytes / (ms * 1e-3) / 1e9,
                "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm, "rate": unit_count / (ms * 1e-3), "rate_unit": unit}

    out = {}
    # motion masks and the dynamic mask
    flow = torch.from_numpy(synth.motion_flow(scene.views, *synth.actor_sphere(scene, 0.05), seed=77)).to(dev)
    bits = torch.empty(max(plan.mask_words, 1), dtype=torch.int32, device=dev)
    dynb = torch.empty(Hh * ((W + 31) // 32), dtype=torch.int32, device=dev)
    ms = timed(lambda: pk.motion_mask(plan, flow, 1.0, 2, bits, r.ws))
    out["motion_mask"] = row(ms, 8 * plan.P + 4 * plan.mask_words, plan.P, "pixels/s")
    out["motion_mask"]["dilate_r"] = 2
    pk.motion_mask(plan, flow, 1.0, 2, bits, r.ws)
    ms = timed(lambda: pk.dynamic_mask(plan, r.records, r.texel, bits, dynb, r.ws))
    out["dynamic_mask"] = row(ms, 24 * plan.pairs + 4 * plan.mask_words, plan.pairs, "pairs/s")
    t = r.texel[:plan.N].long()
    wp = (W + 31) // 32
    dbit = (dynb.long()[(t // W) * wp + (t % W) // 32] >> (t % 32)) & 1
    out["dynamic_mask"]["dynamic_fraction"] = float(dbit.float().mean().item())
    del flow
    # LPO proxy
    if scene.atlas.dtype == np.float32:
        lohi = torch.empty(2 * D, dtype=torch.float32, device=dev)
        codes = torch.empty(F * (D + 3) * Hh * W, dtype=torch.uint8, device=dev)
        texels = F * D * Hh * W
        ms = timed(lambda: pk.lpo_minmax(plan, atlas, occ, lohi, r.ws))
        out["lpo_minmax"] = row(ms, 4 * texels, plan.G, "gaussians/s")
        ms = timed(lambda: pk.lpo_encode(plan, atlas, occ, lohi, codes, r.ws))
        out["lpo_encode"] = row(ms, 4 * texels + F * (D + 3) * Hh * W, plan.G, "gaussians/s")
        ms = timed(lambda: pk.atlas_gather_lpo(plan, codes, pk.api.LPO_CODES, lohi, occ, None, r.soa, r.texel,
                                               r.dynflag, r.ws))
        out["gather_lpo_codes"] = row(ms, plan.G * ((D + 3) + 4 * D), plan.G, "gaussians/s")
        ms = timed(lambda: pk.atlas_gather_lpo(plan, atlas, pk.api.LPO_MASTERS, lohi, occ, None, r.soa, r.texel,
                                               r.dynflag, r.ws))
        out["gather_lpo_fakequant"] = row(ms, plan.G * 8 * D, plan.G, "gaussians/s")
        pk.atlas_gather(plan, atlas, occ, None, r.soa, r.texel, r.dynflag, r.ws)
        del codes
    # Max-K UV pruning of the live set on the base map
    n = plan.N
    soa2 = r.soa.view(plan.D, plan.G)
    cell = torch.empty(n, dtype=torch.int32, device=dev)
    rank = torch.empty_like(cell)
    keep = torch.empty(n, dtype=torch.uint8, device=dev)
    count = torch.empty(W * Hh, dtype=torch.int32, device=dev)
    scratch = pk.uv_max_k(soa2, n, W, Hh, 4, cell, rank, keep, count)
    ms = timed(lambda: pk.uv_max_k(soa2, n, W, Hh, 4, cell, rank, keep, count, scratch))
    out["uv_max_k"] = row(ms, n * (4 * 4 + 4 + 4 + 1 + 8) + W * Hh * 4 * 4, n, "gaussians/s")
    out["uv_max_k"]["map"] = f"{W}x{Hh}, K=4"
    # L1 + D-SSIM objective
    ms = timed(lambda: pk.photo_loss_grad(plan, r.image, target, r.dimage, r.ws, 0.2))
    out["photo_loss_l1_dssim"] = row(ms, 12 * 3 * plan.P, 3 * plan.P, "values/s")
    return out


def ctypes_sizeof_status():
    """Bytes of the device status block read back per step."""
    import ctypes
    from paper_2602_23040_gb300 import _native
    return ctypes.sizeof(_native.DeviceStatus)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--views", type=int, default=0, help="use only the first N cameras (profiling cases)")
    ap.add_argument("--tile", type=int, default=32, choices=[16, 32], help="tile side of the binning")
    ap.add_argument("--ref-window", type=int, default=192)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-view", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--prefetch", type=int, default=6, help="input sets in flight in the end-to-end loop")
    ap.add_argument("--profile", action="store_true", help="short run for a profiler: no extras")
    ap.add_argument("--no-rows", action="store_true", help="skip the rows after the render step")
    ap.add_argument("--with-rows", action="store_true", help="time the rows after the render step even with --profile")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2602_23040_gb300 as pk

    pk.build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    scene = synth.config_scene(args.config, n_views=args.views or None)
    F, D, Hh, W = scene.atlas.shape
    texel_bytes = scene.atlas.dtype.itemsize
    dev = torch.device("cuda", local)
    atlas = torch.from_numpy(scene.atlas).to(dev)
    occ = torch.from_numpy(scene.occ.view(np.int32)).to(dev)
    dyn = None if scene.dyn is None else torch.from_numpy(scene.dyn.view(np.int32)).to(dev)
    target = torch.from_numpy(synth.random_target(scene)).to(dev)
    grad = torch.zeros(F * D * Hh * W, dtype=torch.float32, device=dev)

    # plan sized from a first eager step (re-planned once if the entries overflow)
    r = pk.Renderer(pk.Plan.for_scene(scene, tile=args.tile), dev)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        r.ensure_capacity(atlas, occ, dyn)
        # a profiler run keeps the default options (the ones the tuner picks
        # at this workload) so that its launch sequence stays short and fixed
        batch = r.plan.batch if args.profile else r.autotune(atlas, occ, dyn, target, stream,
                                                             tiles=(args.tile, 48 - args.tile))
        r.l1_step(atlas, occ, dyn, target, grad)
    plan = r.plan
    st = r.status(stream)
    assert st["flags"] == 0, st
    # the evaluation counts (for the ALU roofline) from one pass of the
    # counting variant of the compositing kernels on the same buffers; the
    # timed step runs the variant without counters
    cplan = plan.with_options(count_evals=True)
    with torch.cuda.stream(stream):
        pk.rasterize_fwd_l1(cplan, r.records, r.sorted_vals, r.ranges, target, r.image, r.T, r.n_contrib, r.dimage,
                            r.ws)
        pk.rasterize_bwd(cplan, r.records, r.sorted_vals, r.ranges, r.T, r.n_contrib, r.dimage, r.grad2d, r.ws)
    st = pk.read_status(cplan, r.ws, stream)
    assert st["flags"] == 0, st
    dups, evals_fwd, evals_bwd = int(st["dups"]), int(st["evals_fwd"]), int(st["evals_bwd"])
    del cplan

    # CUDA graph of the whole step
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        r.l1_step(atlas, occ, dyn, target, grad)
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            g.replay()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):      # graph replays launch on the current stream
        e0.record(stream)
        for _ in range(args.steps):
            g.replay()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    mpix = plan.P * world / (ms * 1e-3) / 1e6

    # per-call durations (eager, CUDA events on the launching stream)
    stage_names = ["a1_atlas_gather", "a2_project_and_sh", "a3_bin_and_sort", "a4_rasterize_fwd_l1",
                   "a5_rasterize_bwd", "a6_atlas_scatter_grad"]
    calls = [
        lambda: pk.atlas_gather(plan, atlas, occ, dyn, r.soa, r.texel, r.dynflag, r.ws),
        lambda: pk.project_and_sh(plan, r.soa, r.records, r.ws),
        lambda: pk.bin_and_sort(plan, r.records, r.sorted_vals, r.ranges, r.ws),
        # the step's pair: the forward also clears the 2D gradient records
        lambda: pk.rasterize_fwd_l1_clear(plan, r.records, r.sorted_vals, r.ranges, target, r.image, r.T,
                                          r.n_contrib, r.dimage, r.grad2d, r.ws),
        lambda: pk.rasterize_bwd_accumulate(plan, r.records, r.sorted_vals, r.ranges, r.T, r.n_contrib, r.dimage,
                                            r.grad2d, r.ws),
        lambda: pk.atlas_scatter_grad(plan, r.soa, r.grad2d, r.dynflag if dyn is not None else None, r.texel,
                                      grad, False, r.ws),
    ]
    ksteps = max(1, min(args.steps, 5))
    stage_ms = {n: 0.0 for n in stage_names}
    with torch.cuda.stream(stream):
        for _ in range(ksteps):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)]
            evs[0].record(stream)
            for i, c in enumerate(calls):
                c()
                evs[i + 1].record(stream)
            torch.cuda.synchronize(dev)
            for i, n in enumerate(stage_names):
                stage_ms[n] += evs[i].elapsed_time(evs[i + 1]) / ksteps

    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    n_dyn = plan.G if scene.dyn is None else int(r.dynflag[:plan.N].sum().item()) * F
    bytes_alg = algorithmic_bytes(plan, texel_bytes, dups, n_dyn)
    step_bytes = sum(bytes_alg.values())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", FALLBACK_PEAKS["sm_max_mhz"]))
    alu_peak_tops = sms * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    # dominant single kernel (bin_and_sort is a chain of ~30 kernels and is reported in stages_ms)
    dom = max(("a2_project_and_sh", "a4_rasterize_fwd_l1", "a5_rasterize_bwd", "a6_atlas_scatter_grad"),
              key=lambda n: stage_ms[n])
    t_dom = stage_ms[dom] * 1e-3
    if dom in ("a4_rasterize_fwd_l1", "a5_rasterize_bwd"):
        evals = evals_fwd if dom == "a4_rasterize_fwd_l1" else evals_bwd
        meas = measured_fp32_per_eval(dom)
        # FP32 lane operations per evaluation: the kernel's own, counted by
        # ncu (FADD/FMUL/FFMA, packed forms twice); without a capture of the
        # current sources, the method's ~13 of the scope table
        per_eval = meas["fp32_lane_ops"] if meas else 13.0
        ach = evals * per_eval / t_dom / 1e12
        traffic, tsrc = measured_traffic(dom, dups)
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": alu_peak_tops, "unit": "TOP/s (FP32 lane ops)",
                "frac": ach / alu_peak_tops, "traffic": traffic, "traffic_source": tsrc,
                "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz",
                "fp32_ops_per_evaluation": per_eval,
                "ops_source": meas["source"] if meas else "method count (13 per evaluation), no capture of these sources",
                "evaluations": evals,
                "frac_at_13_ops": evals * 13.0 / t_dom / 1e12 / alu_peak_tops,
                "issue_active_frac": meas["issue_active_pct"] / 100.0 if meas else None,
                "thread_instructions_per_evaluation": meas["thread_inst"] if meas else None,
                "hbm_frac": bytes_alg[dom] / t_dom / 1e9 / hbm}
    else:
        ach = bytes_alg[dom] / t_dom / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "peak_source": f"hbm_gbs ({peak_kind})"}

    out = {
        "metric": METRIC, "value": mpix, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": scene.name, "gaussians": plan.G, "views": plan.V, "pixels": plan.P,
                   "sh_degree": scene.sh_degree, "texels": "fp16" if texel_bytes == 2 else "fp32",
                   "tile": plan.tile, "batch": {"fwd": plan.batch, "bwd": plan.batch_bwd},
                   "staging": {"fwd": plan.stage_fwd, "bwd": plan.stage_bwd},
                   "sort_digit_bits": {"depth": plan.sort_bits_depth, "tile": plan.sort_bits_tile},
                   "tile_trials_ms": getattr(r, "tile_times_ms", None),
                   "pixels_per_thread": {"fwd": 2, "bwd": 4},
                   "tuned_by": "defaults (profiler run)" if args.profile else "pk_autotune", "graph": "whole step in one CUDA graph",
                   "l2": "inputs larger than L2 (atlas %.0f MB, records %.0f MB)" % (
                       scene.atlas.nbytes / 1e6, plan.pairs * 48 / 1e6),
                   "parallelism": f"replica x{world}" if world > 1 else "single GPU"},
        "gaussians_per_s": plan.G * plan.V * world / (ms * 1e-3),
        "hbm_roofline_step": {"algorithmic_bytes": step_bytes, "achieved_gbs": step_bytes / (ms * 1e-3) / 1e9,
                              "peak_gbs": hbm, "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm, "peak": peak_kind},
        "roofline": roof,
        "stages_ms": stage_ms,
        "counts": {"dups": dups, "evals_fwd": evals_fwd, "evals_bwd": evals_bwd, "valid_pairs": int(st["valid_pairs"])},
        "gpu_launches": launches_per_step(plan) * args.steps,
        "clocks": clk,
    }

    if not args.profile and not args.no_e2e:
        # End to end through the public API with host buffers: every step
        # copies its inputs (atlas and target images) from pinned host
        # memory and reads its loss back.  The inputs are prefetched D steps
        # deep (D buffer sets, one captured graph per set): the copies of
        # the next D - 1 steps run on a second stream while this step
        # computes, so an occasional slow host-to-device copy (seen at 85 ms
        # instead of 5.6 ms) lands before its step needs it.
        # the host side runs on the CPUs local to this GPU, so the pinned
        # input buffers are placed (first touch) in the memory nearest to it
        cpus_before, host_cpus = gpu_local_affinity(local)
        h_atlas = torch.from_numpy(scene.atlas).pin_memory()
        h_target = torch.from_numpy(synth.random_target(scene)).pin_memory()
        D = max(2, args.prefetch)
        bufs = [(atlas, target)] + [(torch.empty_like(atlas), torch.empty_like(target)) for _ in range(D - 1)]
        graphs = [g]
        for i in range(1, D):
            gi = torch.cuda.CUDAGraph()
            with torch.cuda.stream(stream):
                r.l1_step(bufs[i][0], occ, dyn, bufs[i][1], grad)      # warm this buffer set
            with torch.cuda.graph(gi, stream=stream):
                r.l1_step(bufs[i][0], occ, dyn, bufs[i][1], grad)
            graphs.append(gi)
        copy_stream = torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(D)]
        ev_done = [torch.cuda.Event() for _ in range(D)]
        ke = max(3, min(2 * args.steps, 40))
        # device time of each step's graph and of each upload, for the breakdown
        g_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ke)]
        u_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ke)]

        def upload(slot, k, timed=True):
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(ev_done[slot])
                if timed:
                    u_ev[k][0].record(copy_stream)
                bufs[slot][0].copy_(h_atlas, non_blocking=True)
                bufs[slot][1].copy_(h_target, non_blocking=True)
                if timed:
                    u_ev[k][1].record(copy_stream)
                ev_in[slot].record(copy_stream)

        # warm-up: one untimed pass over every buffer set (each graph's first
        # replay uploads it to the device; the first copies touch the pinned pages)
        for k in range(D):
            upload(k, 0, timed=False)
            with torch.cuda.stream(stream):
                stream.wait_event(ev_in[k])
                graphs[k].replay()
                ev_done[k].record(stream)
            r.status(stream)
        torch.cuda.synchronize(dev)
        # a host loop that feeds the GPU: the interpreter's cyclic garbage
        # collector is held off while it runs (its passes are host pauses
        # unrelated to the library)
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        for k in range(min(D - 1, ke)):
            upload(k % D, k)
        host = {"replay": [], "upload": [], "status": []}
        step_ms = []
        for k in range(ke):
            slot = k % D
            h0 = time.perf_counter()
            with torch.cuda.stream(stream):
                stream.wait_event(ev_in[slot])
                g_ev[k][0].record(stream)
                graphs[slot].replay()
                g_ev[k][1].record(stream)
                ev_done[slot].record(stream)
            h1 = time.perf_counter()
            if k + D - 1 < ke:
                upload((k + D - 1) % D, k + D - 1)
            h2 = time.perf_counter()
            s = r.status(stream)          # device -> host read of this step's loss (waits for the step)
            h3 = time.perf_counter()
            host["replay"].append((h1 - h0) * 1e3)
            host["upload"].append((h2 - h1) * 1e3)
            host["status"].append((h3 - h2) * 1e3)
            step_ms.append((h3 - h0) * 1e3)
        torch.cuda.synchronize(dev)
        dt = (time.perf_counter() - t0) / ke
        gc.enable()
        gap_ms = statistics.median(g_ev[k][1].elapsed_time(g_ev[k + 1][0]) for k in range(ke - 1))
        graph_ms = statistics.median(a.elapsed_time(b) for a, b in g_ev)
        upload_ms = statistics.median(a.elapsed_time(b) for a, b in u_ev)
        out["e2e"] = {"value": plan.P / dt / 1e6, "unit": UNIT, "ms_per_step": dt * 1e3,
                      "h2d_bytes_per_step": int(h_atlas.numel() * h_atlas.element_size() + h_target.numel() * 4),
                      "d2h_bytes_per_step": int(ctypes_sizeof_status()), "loss": s["loss"],
                      "pipeline": f"inputs prefetched {D} steps deep (one buffer set and graph each); the next "
                                  "steps' copies overlap this step's compute",
                      "graph_ms_per_step": graph_ms, "upload_ms_per_step": upload_ms,
                      "device_gap_between_graphs_ms": gap_ms,
                      "host_ms": {n: statistics.median(v) for n, v in host.items()},
                      "host_step_ms": {"median": statistics.median(step_ms), "max": max(step_ms),
                                       "each": [round(x, 3) for x in step_ms],
                                       "phases_each": {n: [round(x, 3) for x in v] for n, v in host.items()},
                                       "graph_each": [round(a.elapsed_time(b), 3) for a, b in g_ev],
                                       "upload_each": [round(a.elapsed_time(b), 3) for a, b in u_ev]},
                      "steps": ke, "host_cpus": host_cpus}
        if cpus_before is not None:
            os.sched_setaffinity(0, cpus_before)
        del bufs, graphs, h_atlas, h_target

    if not args.profile and not args.no_per_view and rank == 0:
        loop = pk.PerViewLoop.for_scene(scene, dev, tile=plan.tile,
                                        max_dups=int(dups / max(1, plan.V) * 2) + 65536)
        with torch.cuda.stream(stream):
            loop.ensure_capacity(atlas, occ, dyn, target, grad)
        torch.cuda.synchronize(dev)
        kp = max(1, min(args.steps, 3))
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a0.record(stream)
            for _ in range(kp):
                loop.step(atlas, occ, dyn, target, grad)
            a1.record(stream)
        torch.cuda.synchronize(dev)
        pv_ms = a0.elapsed_time(a1) / kp
        ok = all(pk.read_status(p, w)["flags"] == 0 for p, w in zip(loop.plans, loop.ws))
        # the same loop captured in one CUDA graph: its device time without the
        # host's launch gaps, for a like-for-like ratio with the batched graph
        gl = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gl, stream=stream):
            loop.step(atlas, occ, dyn, target, grad)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            gl.replay()
            b0.record(stream)
            for _ in range(kp):
                gl.replay()
            b1.record(stream)
        torch.cuda.synchronize(dev)
        pvg_ms = b0.elapsed_time(b1) / kp
        eager_batched = sum(stage_ms.values())
        out["per_view_loop"] = {"value": plan.P / (pv_ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": pv_ms,
                                "launch": "eager, one view per call sequence", "status_ok": ok,
                                "batched_speedup": pv_ms / ms,
                                "graph_ms_per_step": pvg_ms, "graph_value": plan.P / (pvg_ms * 1e-3) / 1e6,
                                "batched_speedup_same_mode": {
                                    "graph": pvg_ms / ms,
                                    "eager": pv_ms / eager_batched,
                                    "eager_batched_ms": eager_batched,
                                    "note": "graph: both captured whole, device time only; eager: the batched "
                                            "step's per-call sum against the eager per-view loop"}}
        del loop, gl

    if (args.with_rows or not args.profile) and not args.no_rows and rank == 0:
        out["next_rows"] = next_rows(plan, r, scene, atlas, occ, target, stream, dev, hbm)

    if not args.profile and not args.no_cpu_baseline and rank == 0:
        out["cpu_baseline"], win_views, kept = cpu_baseline(scene)
        out["accuracy"] = accuracy_on_windows(scene, win_views, kept, atlas, occ, dyn, dev)
        out["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(args.config, args.views)

    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
