#!/usr/bin/env python3
"""Throughput of the differentiable 6D Gaussian render on GB300.

Workload (the headline configuration): 300,000 6D Gaussians on a noisy unit
shell with strong position-direction coupling, a ring of 8 cameras at
800x800, L1 loss against targets rendered from a seed-perturbed copy of the
scene.  One step = condition_project + bin_sort + raster_fwd_bwd (forward
blend, fused L1 loss and backward blend in one kernel) + project_bwd for all
8 views, i.e. the whole hot path forward and backward.

Arms:
  ours (default)     batched: the 8 views in one launch sequence, replayed
                     as one CUDA graph; also timed: the plain form (the same
                     kernels launched once per view, no graph) and the
                     end-to-end form (host parameters and targets copied in,
                     gradients and loss copied out, every step; the copies of
                     neighbouring steps overlap on two copy streams).
  --impl reference   the FP64 CPU oracle on a bounded sample of the same
                     workload (CPU host cores).

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) execute
independent replicas of the workload, one per GPU ("replicas only": the path
has no exchange step within a step), and report the aggregate.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synth  # noqa: E402

METRIC = "fwd+bwd views/s @800², 300k 6D Gaussians: batched vs plain, same error bound"
UNIT = "views/s"
L2_FLUSH_BYTES = 256 << 20

# Algorithmic work of the fused blend per evaluated (pixel, list entry) pair,
# as the hot-path scope counts it: the forward's 2 subtractions, 6 ops of the
# quadratic form, log2(e) scaling, alpha, clamp, skip test, T update and 3
# colour FMAs (16 FP32 ops + 1 ex2), and the backward's ~50 FP32 ops + 1 MUFU
# (the reciprocal of 1 - alpha) per pair.
FLOPS_PER_PAIR = 16 + 50
MUFU_PER_PAIR = 1 + 1
# A stricter count (FMA = 2 flops, only the work a pair really needs): every
# evaluated pair computes dx, dy and q (10, forward and backward each); a
# compositing pair adds min, 1-alpha, T(1-alpha), w and three colour FMAs (10)
# in the forward, and in the backward the prefix (6), suffix (3), colour grads
# (3), dL/dalpha (15), dq (2), the six geometry grads (12) and the 9-value
# sum over pixels (9) -- 50 -- plus the same 10 as the forward replay.
FLOPS_EVAL_STRICT = 10
FLOPS_COMP_STRICT = 10 + 60
FP32_LANES_PER_SM = 128
SCALE_ROT_BYTES = (21 + 9 + 3) * 4


# Sources of each profiled kernel: roofline "traffic" is taken from the
# kernel's committed ncu summary (profiles/) only while these are unchanged.
KERNEL_SOURCES = {
    "blend_fused_kernel": ["raster.cu"], "blend_bwd_kernel": ["raster.cu"], "blend_fwd_kernel": ["raster.cu"],
    "project_fwd_kernel": ["project.cu", "cond.cuh", "sh.cuh", "mat3.cuh", "stage.cuh"],
    "onesweep_kernel": ["sort.cu"], "emit_expand_kernel": ["sort.cu"], "compact_kernel": ["sort.cu"],
    "geom_bwd_kernel": ["project_bwd.cu", "cond.cuh", "mat3.cuh"],
    "sh_bwd_kernel": ["project_bwd.cu", "cond.cuh", "mat3.cuh", "sh.cuh"],
    "scale_rotation_kernel": ["scale_rotation.cu", "cond.cuh", "mat3.cuh"],
}


def kernel_digest(kernel):
    import hashlib
    h = hashlib.sha1()
    for f in ["common.cuh", "kernels.cuh"] + KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2410_04974_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch from profiles/<kernel>_<workload>.md, or None when
    there is no summary or the kernel's sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    fields = dict(ln.split(": ", 1) for ln in text.splitlines() if ln.startswith(("traffic_bytes_per_launch", "source_digest")))
    if fields.get("source_digest") != kernel_digest(kernel):
        return None
    return int(fields["traffic_bytes_per_launch"])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 200; reference arm 10)")
    ap.add_argument("--warmup", type=int, default=None, help="warm-up steps (default 20; reference arm 3)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2, help="workload index (2 = headline)")
    ap.add_argument("--n", type=int, default=0, help="override the Gaussian count (smaller runs)")
    ap.add_argument("--tile", type=int, nargs=2, default=(16, 16))
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--store-aux", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", action="store_true",
                    help="also time the scale / rotation extraction and the Table-2-shaped inference frames "
                         "(printed as a separate JSON line before the main one)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --tile/--batch as given instead of the autotuner's pick")
    ap.add_argument("--tune-tiles", action="store_true",
                    help="let the autotuner also choose the tile shape (changes the render's tile lists)")
    ap.add_argument("--profile-inference", type=int, default=0,
                    help="run this many single-camera inference frames of the 174,746-point "
                         "Table-2-shaped scene (no timing; for ncu) and exit")
    ap.add_argument("--profile-scale-rotation", action="store_true",
                    help="run the scale / rotation extraction on the 4M-Gaussian tiling of the workload's "
                         "scene three times (no timing; for ncu) and exit")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run this many batched steps eagerly and exit (for ncu)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 10 if args.impl == "reference" else 200
    if args.warmup is None:
        args.warmup = 3 if args.impl == "reference" else 20
    return args


# --------------------------------------------------------------------------
# distributed plumbing
# --------------------------------------------------------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=2)

    def summary(self, busy_mhz_floor=300.0):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        busy = [r for r in rows if r[0] >= busy_mhz_floor] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in busy for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def measure_scale_rotation(l_raw, flush, steps=20, big_n=1 << 22):
    """Time the per-Gaussian scale / rotation extraction on the scene's own
    Gaussians and on a 4M-Gaussian tiling of them (larger than L2).  Algorithmic
    bytes per Gaussian: 21 raw Cholesky floats read, 9 + 3 floats written."""
    import paper_2410_04974_gb300 as sx

    peak = hbm_peak()
    out = {}
    reps = -(-big_n // l_raw.shape[1])
    for name, raw in (("scene", l_raw), ("tiled_4M", l_raw.repeat(1, reps)[:, :big_n].contiguous())):
        n = int(raw.shape[1])
        for _ in range(3):
            sx.scale_rotation(raw)
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, _, status = sx.scale_rotation(raw)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        if int(status.item()) != 0:
            raise RuntimeError(f"scale_rotation status {int(status.item())}")
        ms = sum(times) / len(times)
        gbs = n * SCALE_ROT_BYTES / (ms * 1e-3) / 1e9
        out[name] = {"n": n, "ms": round(ms, 5), "gaussians_per_s": round(n / (ms * 1e-3), 1),
                     "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                                  "frac": round(gbs / peak, 4), "peak_basis": "of measured"}}
    return out


def measure_inference(flush, reps=10, views=synth.TABLE2_TEST_VIEWS):
    """Forward-only frames per second on scenes shaped like the paper's Table 2
    (section 5.2): per scene, the view-independent slice state is cached once,
    then each of `views` test cameras is rendered as its own frame (one
    single-camera inference plan, frames back to back in one CUDA graph).
    L2 is flushed before each timed replay of the `views` frames."""
    import paper_2410_04974_gb300 as sx

    out = []
    for i in range(len(synth.TABLE2_SHAPES)):
        w = synth.table2_workload(i, views=views)
        params = sx.params_to_device(w.scene)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        params["cond_cache"] = sx.condition_cache(params)
        e1.record()
        torch.cuda.synchronize()
        cache_ms = e0.elapsed_time(e1)
        r = sx.Renderer(w.scene.n, w.scene.sh_degree, [w.cameras[0]], inference=True)
        for cam in w.cameras:                      # size the duplicate capacity for every view
            r.set_cameras([cam])
            r.forward(params)
        imgs = [r.new_images() for _ in w.cameras]

        def frames():
            for v, cam in enumerate(w.cameras):
                r.set_cameras([cam])
                r.condition_project(params)
                r.bin_sort()
                r.raster_fwd(imgs[v])

        r.status.zero_()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            frames()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            frames()
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        r.raise_status()
        times = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            graph.replay()
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        r.raise_status()
        ms_frame = sum(times) / len(times) / len(w.cameras)
        # per-stage split of one frame (eager launches)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        split = np.zeros(3)
        for cam in w.cameras:
            r.set_cameras([cam])
            ev[0].record()
            r.condition_project(params)
            ev[1].record()
            r.bin_sort()
            ev[2].record()
            r.raster_fwd(imgs[0])
            ev[3].record()
            torch.cuda.synchronize()
            split += [ev[k].elapsed_time(ev[k + 1]) for k in range(3)]
        split /= len(w.cameras)
        # all test views as one batched inference plan
        rb = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras, inference=True)
        img_b = rb.forward(params)
        tb = []
        for _ in range(max(3, reps // 2)):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            rb.condition_project(params)
            rb.bin_sort()
            rb.raster_fwd(img_b)
            b.record()
            torch.cuda.synchronize()
            tb.append(a.elapsed_time(b))
        rb.raise_status()
        ms_batch = sum(tb) / len(tb)
        name, n, side_px, kind, paper_fps = synth.TABLE2_SHAPES[i]
        out.append({"workload": name, "n_gaussians": n, "resolution": f"{side_px}x{side_px}",
                    "fps": round(1000.0 / ms_frame, 1), "ms_per_frame": round(ms_frame, 4),
                    "stage_ms": {"condition_project": round(split[0], 4), "bin_sort": round(split[1], 4),
                                 "raster_fwd": round(split[2], 4)},
                    "batched_views_per_s": round(len(w.cameras) * 1000.0 / ms_batch, 1),
                    "cache_build_ms": round(cache_ms, 4),
                    "duplicates_last_view": int(r.counts()[1]),
                    "paper_fps_6dgs": paper_fps})
        del r, rb, imgs, img_b, graph, params
        torch.cuda.empty_cache()
    return {"frames_per_scene": views, "l2": "flushed before each timed replay of the frames",
            "paper_hardware": "not named in the paper", "scenes": out}


def host_copy_rates(dev, nbytes=256 << 20, reps=3):
    """Pinned host <-> device copy rates (GB/s, best of `reps`), the bound on
    the end-to-end figure's copies."""
    host = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    buf = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {}
    for name, fn in (("h2d", lambda: buf.copy_(host, non_blocking=True)),
                     ("d2h", lambda: host.copy_(buf, non_blocking=True))):
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = round(nbytes / (best * 1e-3) / 1e9, 1)
    return out


def measure_alu_peaks(sms, reps=5):
    """Achieved FP32 FMA (TFLOP/s) and MUFU ex2 (Tops/s) rates of the library's
    saturating probe kernels, best of `reps`, at the GPU's current clocks."""
    import ctypes

    import paper_2410_04974_gb300 as sx

    lib = sx._lib.load()
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    res = {}
    for kind, iters, name, ops_per in ((0, 4096, "fp32_fma_tflops", 2.0), (1, 512, "mufu_ex2_tops", 1.0)):
        best = float("inf")
        for _ in range(reps + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sx._lib.check(lib.sixdgs_peak_probe(kind, iters, ctypes.c_void_p(out.data_ptr()), blocks, stream),
                          "sixdgs_peak_probe")
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        res[name] = round(blocks * 256 * iters * 8 * ops_per / (best * 1e-3) / 1e12, 2)
    return res


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def launches_per_frame(plan, n_cams):
    """Kernels of ours one fwd+bwd frame launches: camera upload (one per 48
    cameras), projection, compaction, depth passes, emission (scan + expand),
    tile passes, ranges, fused blend forward + L1 + blend backward, SH
    backward, geometry backward."""
    return (n_cams + 47) // 48 + 1 + 1 + plan.depth_passes + 2 + plan.tile_passes + 1 + 1 + 1 + 1

def build_inputs(args):
    w = synth.make_workload(args.config, n_override=args.n or None)
    target_scene = synth.perturb(w.scene, synth.target_seed(args.config))
    return w, target_scene


def run_ours(args, world, rank, local):
    import paper_2410_04974_gb300 as sx

    from paper_2410_04974_gb300 import autotune

    dev = torch.device("cuda", local)
    w, tscene = build_inputs(args)
    cams = w.cameras
    V = len(cams)
    params = sx.params_to_device(w.scene, dev)
    base_kw = dict(lambda_opa=w.lambda_opa, bg=w.bg, store_aux=args.store_aux)
    tuned = None
    if args.no_autotune or args.profile_steps:
        kw = dict(tile=tuple(args.tile), batch=args.batch, persistent=False, **base_kw)
    else:
        tiles = ((16, 16), (16, 8), (32, 8), (8, 16), (32, 16)) if args.tune_tiles else (tuple(args.tile),)
        space = autotune.candidate_space(tiles=tiles, batches=(256, 512, 1024), persistent=(True, False))
        tuned = autotune.tune(params, w.scene.n, w.scene.sh_degree, cams, space=space, **base_kw)
        kw = dict(tile=tuple(tuned["tile"]), batch=tuned["batch"], persistent=tuned["persistent"], **base_kw)
    # targets: render the perturbed scene once (untimed)
    rt = sx.Renderer(tscene.n, tscene.sh_degree, cams, **kw)
    targets = rt.forward(sx.params_to_device(tscene, dev))
    torch.cuda.synchronize()
    del rt

    r = sx.Renderer(w.scene.n, w.scene.sh_degree, cams, **kw)
    images = r.forward(params)                       # sizes the duplicate capacity
    torch.cuda.synchronize()
    cap = r.plan.dup_capacity
    gimg = torch.empty_like(images)
    grads = r.new_grads(params)

    def step(rr=r, out_grads=grads):
        rr.status.zero_()
        rr.loss.zero_()
        rr.condition_project(params)
        rr.bin_sort()
        rr.raster_fwd_bwd(images, targets, gimg, rr.loss)
        rr.project_bwd(params, out_grads)

    step()
    torch.cuda.synchronize()
    r.raise_status()
    counts = r.counts()

    if args.profile_steps:
        for _ in range(args.profile_steps):
            step()
        torch.cuda.synchronize()
        r.raise_status()
        if rank == 0:
            print(json.dumps({"profile_steps": args.profile_steps, "counts": counts.tolist()}))
        return

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # ---- batched: one CUDA graph per step ----
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(3):
            step()
    torch.cuda.current_stream(dev).wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    r.raise_status()

    def timed(fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        barrier(world)
        torch.cuda.synchronize()
        for e0, e1 in evs:
            flush.zero_()
            e0.record()
            fn()
            e1.record()
        torch.cuda.synchronize()
        barrier(world)
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_id = vis.split(",")[local].strip() if vis else str(local)
    with ClockSampler(smi_id) as clocks:
        t_batched = timed(graph.replay, args.steps)
    r.raise_status()
    ms_batched = max_over_ranks(sum(t_batched) / len(t_batched), world)
    img_batched = images.clone()
    grads_batched = {k: v.clone() for k, v in grads.items()}
    loss_batched = float(r.loss.item())

    # ---- per-stage breakdown (eager launches, same flush discipline) ----
    stage_names = ["condition_project", "bin_sort", "raster_fwd_bwd", "project_bwd"]

    def staged():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(stage_names) + 1)]
        r.status.zero_()
        r.loss.zero_()
        ev[0].record()
        r.condition_project(params)
        ev[1].record()
        r.bin_sort()
        ev[2].record()
        r.raster_fwd_bwd(images, targets, gimg, r.loss)
        ev[3].record()
        r.project_bwd(params, grads)
        ev[4].record()
        return ev

    stage_steps = max(5, min(args.steps, 50))
    all_ev = []
    for _ in range(3):
        staged()
    torch.cuda.synchronize()
    for _ in range(stage_steps):
        flush.zero_()
        all_ev.append(staged())
    torch.cuda.synchronize()
    stages = {name: sum(ev[i].elapsed_time(ev[i + 1]) for ev in all_ev) / stage_steps
              for i, name in enumerate(stage_names)}

    # ---- plain: same kernels, one camera at a time, no graph ----
    plain = None
    equiv = None
    if not args.no_plain:
        # one single-camera plan per distinct resolution; the loss is normalised
        # over the whole batch so losses and gradients equal the batched ones
        plain_r = {}
        for c in cams:
            key = (c.width, c.height)
            if key not in plain_r:
                plain_r[key] = sx.Renderer(w.scene.n, w.scene.sh_degree, [c], loss_norm=3.0 * r.total_pixels, **kw)
        offs = np.cumsum([0] + [3 * h * wd for (h, wd) in r.sizes])
        per_view = [slice(int(offs[v]), int(offs[v + 1])) for v in range(V)]
        grads_p = r.new_grads(params)
        loss_p = torch.zeros(1, dtype=torch.float64, device=dev)

        def plain_step():
            loss_p.zero_()
            for rr in plain_r.values():
                rr.status.zero_()
            for v in range(V):
                rp = plain_r[(cams[v].width, cams[v].height)]
                rp.set_cameras([cams[v]])
                sl = per_view[v]
                rp.condition_project(params)
                rp.bin_sort()
                rp.raster_fwd_bwd(images[sl], targets[sl], gimg[sl], loss_p)
                rp.project_bwd(params, grads_p, accumulate=v > 0)

        for _ in range(max(3, args.warmup // 2)):
            plain_step()
        torch.cuda.synchronize()
        for rr in plain_r.values():
            rr.raise_status()
        t_plain = timed(plain_step, max(10, args.steps // 4))
        for rr in plain_r.values():
            rr.raise_status()
        ms_plain = max_over_ranks(sum(t_plain) / len(t_plain), world)
        rp0 = next(iter(plain_r.values()))
        plain = {"value": V * 1000.0 / ms_plain * world, "unit": UNIT, "ms_per_step": ms_plain,
                 "launches_per_step": V * launches_per_frame(rp0.plan, 1), "graph": False}
        g_rel = {k: float((grads_p[k] - grads_batched[k]).norm() / grads_batched[k].norm().clamp_min(1e-30))
                 for k in grads_p}
        equiv = {"image_max_abs": float((images - img_batched).abs().max()),
                 "loss_abs": abs(float(loss_p.item()) - loss_batched),
                 "grad_rel_l2_max": max(g_rel.values())}
        del plain_r

    # ---- end to end through the C ABI with host buffers ----
    # Every step copies its inputs (scene parameters, target images) in from
    # pinned host memory and its results (gradients, loss) out to pinned host
    # memory, inside the timed region.  "sequential": copy in, step, copy out
    # on one stream.  Pipelined (the reported e2e): step k+1's inputs are
    # copied in on one copy stream while step k computes, and step k's results
    # are copied out on another while step k+1 computes (double-buffered
    # device staging), as a training loop's data pipeline would run.
    e2e = None
    if not args.no_e2e:
        main = torch.cuda.current_stream(dev)
        host = {k: v.detach().cpu().pin_memory() for k, v in params.items()}
        host_t = targets.cpu().pin_memory()
        host_g = [{k: torch.empty_like(v, device="cpu").pin_memory() for k, v in grads.items()} for _ in range(2)]
        host_loss = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
        h2d = sum(v.numel() * 4 for v in host.values()) + host_t.numel() * 4
        d2h = sum(v.numel() * 4 for v in host_g[0].values()) + 8

        def e2e_step():
            for k in params:
                params[k].copy_(host[k], non_blocking=True)
            targets.copy_(host_t, non_blocking=True)
            graph.replay()
            for k in grads:
                host_g[0][k].copy_(grads[k], non_blocking=True)
            host_loss[0].copy_(r.loss, non_blocking=True)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        t_seq = timed(e2e_step, max(10, args.steps // 4))
        ms_seq = max_over_ranks(sum(t_seq) / len(t_seq), world)

        # a second set of step buffers with its own captured graph, so that
        # step k+1's inputs can be copied in while step k computes on the other
        # set, and step k's gradients copied out while step k+1 computes
        params_b = {k: v.clone() for k, v in params.items()}
        targets_b = targets.clone()
        grads_b = r.new_grads(params)

        def step_b():
            r.status.zero_()
            r.loss.zero_()
            r.condition_project(params_b)
            r.bin_sort()
            r.raster_fwd_bwd(images, targets_b, gimg, r.loss)
            r.project_bwd(params_b, grads_b)

        side_b = torch.cuda.Stream(dev)
        side_b.wait_stream(main)
        with torch.cuda.stream(side_b):
            for _ in range(2):
                step_b()
        main.wait_stream(side_b)
        graph_b = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_b):
            step_b()
        torch.cuda.synchronize()
        sets = [(params, targets, grads, graph), (params_b, targets_b, grads_b, graph_b)]
        loss_stage = [torch.zeros_like(r.loss) for _ in range(2)]
        h2d_s, d2h_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

        def pipelined(K):
            ev = {n: [torch.cuda.Event() for _ in range(2)] for n in ("in_ready", "in_free", "done", "out_free")}

            def copy_in(k):
                b = k % 2
                p_, t_ = sets[b][0], sets[b][1]
                with torch.cuda.stream(h2d_s):
                    h2d_s.wait_event(ev["in_free"][b])       # step k-2 no longer reads this set
                    for name in p_:
                        p_[name].copy_(host[name], non_blocking=True)
                    t_.copy_(host_t, non_blocking=True)
                    ev["in_ready"][b].record(h2d_s)

            h2d_s.wait_stream(main)
            d2h_s.wait_stream(main)
            copy_in(0)
            for k in range(K):
                b = k % 2
                if k + 1 < K:
                    copy_in(k + 1)
                g_, gr = sets[b][2], sets[b][3]
                main.wait_event(ev["in_ready"][b])
                main.wait_event(ev["out_free"][b])           # step k-2's gradients are out
                gr.replay()
                loss_stage[b].copy_(r.loss, non_blocking=True)
                ev["in_free"][b].record(main)
                ev["done"][b].record(main)
                with torch.cuda.stream(d2h_s):
                    d2h_s.wait_event(ev["done"][b])
                    for name in g_:
                        host_g[b][name].copy_(g_[name], non_blocking=True)
                    host_loss[b].copy_(loss_stage[b], non_blocking=True)
                    ev["out_free"][b].record(d2h_s)
            main.wait_stream(d2h_s)
            main.wait_stream(h2d_s)

        pipelined(3)
        torch.cuda.synchronize()
        k_e2e = max(10, args.steps // 4)
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        pipelined(k_e2e)
        e1.record()
        torch.cuda.synchronize()
        barrier(world)
        ms_e2e = max_over_ranks(e0.elapsed_time(e1) / k_e2e, world)
        r.raise_status()
        last = (k_e2e - 1) % 2
        e2e_check = max(float((host_g[last][k] - grads_batched[k].cpu()).norm() /
                              grads_batched[k].cpu().norm().clamp_min(1e-30)) for k in grads_batched)
        e2e = {"value": V * 1000.0 / ms_e2e * world, "unit": UNIT, "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "mode": "pipelined: step k+1's host-to-device copies and step k-1's device-to-host copies "
                       "overlap step k's compute (two copy streams, two buffer sets with one captured graph "
                       "each); the working set is larger than L2",
               "grad_rel_l2_vs_batched": e2e_check,
               "sequential": {"value": V * 1000.0 / ms_seq * world, "ms_per_step": ms_seq,
                              "l2": "flushed between steps"},
               "host_copy_gbs": host_copy_rates(dev)}

    # ---- roofline of the dominant kernel ----
    rc = sx.Renderer(w.scene.n, w.scene.sh_degree, cams, count_pairs=True, **kw)
    rc.forward(params)
    torch.cuda.synchronize()
    n_eval, n_comp, n_warp = [int(x) for x in rc.pair_counts()]
    del rc
    clk = clocks.summary()
    dom = "raster_fwd_bwd"
    dom_ms = stages[dom]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_clock = float(clk["sm_mhz"] or 2070.0)
    peak = sms * FP32_LANES_PER_SM * 2 * peak_clock * 1e6 / 1e12
    achieved = n_eval * FLOPS_PER_PAIR / (dom_ms * 1e-3) / 1e12
    strict = (n_eval * 2 * FLOPS_EVAL_STRICT + n_comp * FLOPS_COMP_STRICT) / (dom_ms * 1e-3) / 1e12
    kernel = "blend_fused_kernel"
    measured = measure_alu_peaks(sms)
    mufu = n_eval * MUFU_PER_PAIR / (dom_ms * 1e-3) / 1e12
    t_sorted = sorted(t_batched)
    roofline = {"bound": "alu", "kernel": kernel, "achieved": round(achieved, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": profiled_traffic(kernel, w.name),
                "count": f"{FLOPS_PER_PAIR} FP32 ops + {MUFU_PER_PAIR} MUFU per evaluated (pixel, entry) pair",
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {peak_clock:.0f} MHz",
                "kernel_ms": round(dom_ms, 4), "pairs_evaluated": n_eval, "pairs_compositing": n_comp,
                "warp_entries": n_warp,
                "frac_strict_count": round(strict / peak, 4),
                "frac_of_measured_fp32": round(achieved / measured["fp32_fma_tflops"], 4),
                "mufu_tops": round(mufu, 3), "frac_of_measured_mufu": round(mufu / measured["mufu_ex2_tops"], 4),
                "measured_alu_peaks": measured,
                "step_ms": {"min": round(t_sorted[0], 4), "median": round(statistics.median(t_sorted), 4),
                            "p90": round(t_sorted[min(len(t_sorted) - 1, int(0.9 * len(t_sorted)))], 4),
                            "max": round(t_sorted[-1], 4)},
                "stages_ms": {k: round(v, 4) for k, v in stages.items()},
                "batched_vs_plain": None if plain is None else {
                    "plain_views_per_s": round(plain["value"], 1), "plain_ms_per_step": round(plain["ms_per_step"], 4),
                    "speedup": round(plain["ms_per_step"] / ms_batched, 3), **{k: float(f"{v:.3g}") for k, v in equiv.items()}},
                "launch": {"batch": kw["batch"], "persistent": bool(kw["persistent"]), "visible_pairs": int(counts[0]),
                           "duplicates": int(counts[1])}}

    # ---- optional: scale / rotation extraction and inference frames ----
    if args.extras and rank == 0:
        extras = {"scale_rotation": measure_scale_rotation(params["l_raw"], flush),
                  "inference": measure_inference(flush)}
        print(json.dumps({"extras": extras}))

    # ---- CPU baseline: the oracle on whole views (rank 0) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(w)

    value = V * 1000.0 / ms_batched * world
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_batched, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, kw["tile"], world),
        "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
        "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "gpu_launches": launches_per_frame(r.plan, V) * args.steps,
        "megapixels_per_s": round(r.total_pixels * world / (ms_batched * 1e-3) / 1e6, 1),
        "loss": loss_batched,
        "autotuned": None if tuned is None else {k: tuned[k] for k in ("tile", "batch", "persistent", "ms", "cached")},
    }
    if rank == 0:
        print(json.dumps(line))


def workload_config(w, tile, world):
    """The workload description, the same in both arms."""
    cams = w.cameras
    return {"workload": w.name, "n_gaussians": w.scene.n, "views": len(cams),
            "resolution": sorted({f"{c.width}x{c.height}" for c in cams}), "tile": list(tile),
            "sh_degree": w.scene.sh_degree, "loss": "L1 vs targets of a perturbed scene",
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "GPU arm: 256 MiB written between timed steps (flush); CPU arm: whole views"}


# --------------------------------------------------------------------------
# the oracle (CPU baseline and reference arm)
# --------------------------------------------------------------------------

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_view_seconds(w, v, seed=0):
    """Seconds the FP64 oracle takes for one whole view of the training step:
    the slice, colour and projection of every Gaussian, then forward and
    backward (autograd) of every occupied 16x16 tile with a seeded dL/dI."""
    from oracle import sixdgs_oracle as O

    st = O.Settings(tile_w=16, tile_h=16, lambda_opa=w.lambda_opa, bg=w.bg)
    cam = w.cameras[v % len(w.cameras)]
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    with torch.no_grad():
        prep = O.prepare_view(O.to_params(w.scene), w.scene.sh_degree, cam, st)
    tx, ty = O.tile_grid(cam, st)
    rect = prep.rect.numpy()[prep.valid.numpy()]
    occupied = np.zeros((ty, tx), bool)
    for x0, x1, y0, y1 in rect:
        occupied[y0:y1, x0:x1] = True
    tiles = [(int(x), int(y)) for y, x in np.argwhere(occupied)]
    g = rng.normal(size=(3, cam.height, cam.width)).astype(np.float32)
    O.gradients(w.scene, [cam], [g], st, tiles=[tiles])
    return time.perf_counter() - t0, len(tiles)


def oracle_baseline(w):
    """Views/s of the FP64 oracle on whole views of the workload: two views
    with all of the process's threads, one view with a single thread."""
    threads = torch.get_num_threads()
    secs, tiles = zip(*(oracle_view_seconds(w, v, seed=v) for v in range(2)))
    value = 2.0 / sum(secs)
    torch.set_num_threads(1)
    try:
        one, _ = oracle_view_seconds(w, 2, seed=2)
    finally:
        torch.set_num_threads(threads)
    return {"value": round(value, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"2 whole views of {w.name}, fwd+bwd of all {tiles[0]}+{tiles[1]} occupied tiles",
            "cpu_model": cpu_model(), "seconds_measured": round(sum(secs), 2),
            "single_thread": {"value": round(1.0 / one, 6), "cores": 1, "sample": "1 whole view",
                              "seconds_measured": round(one, 2)}}


def run_reference(args, world, rank):
    """The oracle as the reference arm: every step is one whole view of the
    workload (cameras in turn), forward and backward, on the host cores."""
    if rank != 0:
        return
    w, _ = build_inputs(args)
    times = []
    tiles = 0
    for k in range(args.warmup + args.steps):
        dt, tiles = oracle_view_seconds(w, k, seed=k)
        if k >= args.warmup:
            times.append(dt)
    view_s = float(np.mean(times))
    value = 1.0 / view_s
    threads = torch.get_num_threads()
    cpu = {"value": round(value, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"1 whole view per step ({tiles} occupied tiles in the last), cameras in turn",
           "cpu_model": cpu_model()}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(view_s * 1000.0, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, (16, 16), world),
            "cpu_baseline": cpu, "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def profile_inference(frames):
    """Inference frames of one Table-2-shaped scene, untimed, for ncu captures."""
    import paper_2410_04974_gb300 as sx

    w = synth.table2_workload(4)
    params = sx.params_to_device(w.scene)
    params["cond_cache"] = sx.condition_cache(params)
    r = sx.Renderer(w.scene.n, w.scene.sh_degree, [w.cameras[0]], inference=True)
    img = r.new_images()
    for f in range(frames):
        r.set_cameras([w.cameras[f % len(w.cameras)]])
        img = r.forward(params)
    torch.cuda.synchronize()
    print(json.dumps({"profile_inference": frames, "workload": w.name, "counts": r.counts().tolist()}))


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.profile_inference:
        profile_inference(args.profile_inference)
        return
    if args.profile_scale_rotation:
        import paper_2410_04974_gb300 as sx

        w, _ = build_inputs(args)
        raw = torch.as_tensor(w.scene.l_raw).cuda()
        big = raw.repeat(1, -(-(1 << 22) // raw.shape[1]))[:, :1 << 22].contiguous()
        for _ in range(3):
            _, _, status = sx.scale_rotation(big)
        torch.cuda.synchronize()
        print(json.dumps({"profile_scale_rotation": int(big.shape[1]), "status": int(status.item())}))
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        if not torch.cuda.is_available():
            raise SystemExit("bench.py (ours) needs a CUDA GPU")
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
