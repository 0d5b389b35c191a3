#!/usr/bin/env python
"""Benchmark of the differentiable tile rasterizer: 1080p forward+backward frames/s at 3M
Gaussians (synthetic large unbounded scene, SH degree 3, 1920x1080).

One step = one pass of the whole hot path over one frame: gs_preprocess, gs_bin_sort,
gs_render_forward, gs_render_backward (tiles, then Gaussians).  Inputs are resident in HBM
for ``value``; ``e2e`` repeats the measurement with the inputs in pinned host memory and the
image and gradients copied back every step.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the only reference this project has) on the
same frame, one whole frame per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p fwd+bwd frames/s at 3M Gaussians"
UNIT = "frames/s"
WORKLOAD = "large unbounded scene: 3M Gaussians, SH degree 3, 1920x1080, forward+backward"

# The render kernels' roofline is an ALU one; its peak is measured on the GPU at the start of
# every run (measure_alu_peaks: FP32 FMA chains, gs_peak_fma).  The nominal figure, for
# context: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz.
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
ALU_NOMINAL_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
# FP32 flops per evaluated (pixel, Gaussian) pair on the path every evaluation takes
# (offset 2, quadratic form 7, exp 2, opacity 1, clamp 1, threshold 1) and extra flops of a
# blended pair (forward: transmittance 2, weight 1, colour 6; backward: recovery 5,
# colour gradient 3, alpha gradient 7, R update 9, conic/mean/opacity gradients 15).
FLOPS_EVAL = 14
FLOPS_BLEND_FWD = 9
FLOPS_BLEND_BWD = 39

CONFIG3_N = 3_000_000
KERNEL_NAMES = {"preprocess": "k_preprocess_t", "render_forward": "k_render_forward_t",
                "render_backward_tiles": "k_render_backward_t",
                "render_backward_gaussians": "k_preprocess_backward_t"}
# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one launch of each
# single-kernel stage on the 3M-Gaussian 1080p frame, taken from a capture of the current
# kernel; a stage without such a capture reports None.
TRAFFIC = {"render_backward_tiles": 107_670_016, "render_forward": 70_443_008}


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# Measured ALU peaks (denominators of the render kernels' roofline)
# ------------------------------------------------------------------------------------------
def measure_alu_peaks(dev, seconds: float = 0.4) -> dict:
    """FP32 FMA and 2^x (ex2.approx.ftz.f32) throughput of this GPU: gs_peak_fma / gs_peak_ex2 with two 1024-thread
    blocks per SM, each timed with CUDA events over about `seconds`, clocks sampled meanwhile."""
    import torch
    from paper_2308_04079_gb300 import _abi
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 2 * sms
    sink = torch.zeros(blocks, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {"blocks": blocks, "threads": 1024, "sms": sms}
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    time.sleep(0.3)
    for name, fn in (("fma", _abi.gs_peak_fma), ("ex2", _abi.gs_peak_ex2)):
        iters = 2000
        fn(blocks, iters, sink.data_ptr(), stream.cuda_stream)            # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(blocks, iters, sink.data_ptr(), stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        iters = max(2000, int(iters * seconds / max(a.elapsed_time(b) * 1e-3, 1e-6)))
        a.record(stream)
        fn(blocks, iters, sink.data_ptr(), stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        ops = _abi.gs_peak_ops(blocks, iters)
        out[name] = {"ms": round(ms, 3), "ops": ops, "rate_per_s": ops / (ms * 1e-3)}
    clocks = sampler.stop()
    out["fma_tflops"] = round(2 * out["fma"]["rate_per_s"] / 1e12, 2)
    out["ex2_gops"] = round(out["ex2"]["rate_per_s"] / 1e9, 1)
    out["clocks"] = clocks
    if clocks.get("sm_mhz"):
        # per-clock rates: 152 SMs x 128 lanes x 2 would be 38912 flops per cycle
        out["fma_flops_per_cycle"] = round(2 * out["fma"]["rate_per_s"] / (clocks["sm_mhz"] * 1e6), 1)
        out["ex2_per_cycle"] = round(out["ex2"]["rate_per_s"] / (clocks["sm_mhz"] * 1e6), 1)
    for k in ("fma", "ex2"):
        out[k]["rate_per_s"] = round(out[k]["rate_per_s"], 1)
    assert float(sink.abs().sum().item()) == 0.0
    return out


# ------------------------------------------------------------------------------------------
# Our arm
# ------------------------------------------------------------------------------------------
def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks (the slowest rank's time); x itself for one rank."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


def workload_config(n, cam, tile, world) -> dict:
    """The workload a step processes; both arms print the same dict."""
    return {"workload": WORKLOAD if n == CONFIG3_N else f"{WORKLOAD} (subsampled to {n} Gaussians)",
            "gaussians": n, "width": cam.width, "height": cam.height, "sh_degree": 3,
            "tile": f"{tile[0]}x{tile[1]}",
            "l2": "inputs larger than L2 (708 MB of Gaussian parameters read per step)",
            "parallelism": f"replicas x{world}"}


def row_sort(layout) -> bool:
    """Two-phase frames up to 255 tile columns take the row-segmented tile sort."""
    return bool(layout.depth_passes) and layout.tiles_x <= 255


def launches_per_step(layout) -> int:
    """Kernels one step launches: preprocess; binning = two-phase: depth histogram + depth
    passes + one segment pass (count, scan and records), then either sort-prepare + row passes
    over the records + column count + tile scan + column pass (key_passes = row passes + 1) or
    emit + sort-prepare + instance passes + ranges; KEY64: count + pair scan + segment write +
    emit + sort-prepare + instance passes + ranges; every schedule starts with one clear kernel
    (its four zeroed regions) and ends with the tile order of the render passes; forward;
    backward tiles after one clear kernel (accumulators and counter); backward Gaussians.  Both
    two-phase forms launch 5 + key_passes binning kernels after the depth sort."""
    if layout.depth_passes:
        binning = (1 + layout.depth_passes) + 1 + 3 + layout.key_passes
    else:
        binning = 3 + 3 + layout.key_passes
    return 1 + (1 + binning + 1) + 1 + (1 + 1) + 1


def byte_model(n, n_vis, K, segs, P, tiles, sh_floats, layout):
    """Algorithmic DRAM bytes per launch of each stage: what the stage must read and write
    once, with the measured visible count, instance count K and segment count."""
    b = {}
    # read mu, s, q, o (44 B) for every Gaussian and the SH rows (sh_floats x 4 B) of visible
    # ones; write mean (16), depth (4), conic+opacity (16), rgb (16), radius (4), tau (4)
    b["preprocess"] = n * (44 + 60) + n_vis * sh_floats * 4
    key_bytes = 4 if layout.depth_passes else 8
    # depth sort (two-phase): histogram read of depth+radius, then per pass read+write of
    # (key, value); scan: per visible Gaussian read order, radius, mean, conic, tau (44 B),
    # write 12 B per segment record; emit: read the records, write K (key, value); instance
    # sort passes: read+write K (key, value); ranges: 8 B per tile
    depth_sort = (8 * n + layout.depth_passes * 16 * n) if layout.depth_passes else 0
    if row_sort(layout):
        # row sort: 8 B per (row key, Gaussian) record written, read + written by each row
        # pass, read by the column count (4 B) and the column pass (8 B); tile counts and
        # ranges 12 B per tile; the column pass writes K (tile id, Gaussian)
        rp = layout.key_passes - 1
        b["bin_sort"] = depth_sort + n_vis * 44 + segs * (8 + rp * 16 + 4 + 8) + tiles * 12 + K * 8
    else:
        b["bin_sort"] = depth_sort + n_vis * 44 + segs * 12 * 2 + K * (key_bytes + 4) \
            + layout.key_passes * 2 * K * (key_bytes + 4) + tiles * 8
    # per instance one value read and one gathered splat (mean 16 + conic 16 + rgb 16 = 48 B;
    # the gather of a splat is counted once per instance, i.e. L2 reuse across tiles ignored);
    # per pixel write rgb, T, last (20 B)
    b["render_forward"] = K * (4 + 48) + P * 20 + tiles * 8
    # per instance value + splat gather; per pixel read dL/dC, T, last (20 B); per visible
    # Gaussian 48 B of accumulators written (atomics) once
    b["render_backward_tiles"] = K * (4 + 48) + P * 20 + tiles * 8 + n_vis * 48
    # per Gaussian read parameters (44 B) and, for visible ones, SH rows, accumulators (48 B)
    # and screen-space state (36 B); write every gradient (236 B) and the mean2d gradient (8 B)
    b["render_backward_gaussians"] = n * (44 + 236 + 8) + n_vis * (sh_floats * 4 + 48 + 36)
    return b


def run_ours(args, rank, world, local_rank):
    import torch
    import synthetic as S
    from paper_2308_04079_gb300 import Frame, GaussianTensors, _abi, make_config
    from paper_2308_04079_gb300 import build as gbuild

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if gbuild.needs_build():
        gbuild.build()
    g, cam, bg, dimg = S.config3(n=args.gaussians, k=1 + rank)
    bg = tuple(float(x) for x in bg)
    gt = GaussianTensors.from_numpy(g, device=dev).prepared()
    d_dimg = torch.from_numpy(dimg).to(dev)
    cfg = make_config(sort_mode=args.sort_mode)
    fr = Frame(gt.n, cam, cfg, device=dev)
    fr.ensure_binned(gt)
    K = int(fr.last_status.num_instances)
    fr = Frame(gt.n, cam, cfg, capacity=int(K * 1.15) + 4096, device=dev)
    img, T, last = fr.outputs()
    grads = fr.new_grads(gt)
    stream = torch.cuda.current_stream()
    stages = ["preprocess", "bin_sort", "render_forward", "render_backward_tiles", "render_backward_gaussians"]

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        fr.preprocess(gt)
        if ev is not None:
            ev[1].record(stream)
        fr.bin_sort()
        if ev is not None:
            ev[2].record(stream)
        fr.render_forward(bg, img, T, last)
        if ev is not None:
            ev[3].record(stream)
        fr.render_backward_tiles(bg, d_dimg, T, last)
        if ev is not None:
            ev[4].record(stream)
        fr.render_backward_gaussians(gt, grads)
        if ev is not None:
            ev[5].record(stream)

    peaks = measure_alu_peaks(dev)
    for _ in range(args.warmup):
        step()
    code, st = fr.status()
    if code not in (_abi.GS_OK, _abi.GS_ERR_NUMERIC):
        raise RuntimeError(f"warm-up step failed: {_abi.status_string(code)}")
    n_vis, K = int(st.num_visible), int(st.num_instances)
    sum_last = float(last.to(torch.float64).sum().item())
    blended = int(st.blended_pairs)
    segs = int(st.num_segments)

    # per-launch times of the binning stage (outside the timed region; the stage re-bins the
    # preprocessed frame): median of 5 runs, with the keys each sorting pass moves
    runs = [fr.bin_sort_timed() for _ in range(5)]
    bin_launches = []
    for i, (label, _) in enumerate(runs[0]):
        ms = float(np.median([r[i][1] for r in runs]))
        keys = {"depth radix pass": gt.n, "row radix pass": segs, "instance radix pass": K, "column pass": K,
                "segment pass": n_vis, "column count": segs}.get(label)
        e = {"launch": label, "ms": round(ms, 4)}
        if keys:
            e["keys"] = int(keys)
            e["keys_per_s"] = round(keys / (ms * 1e-3), 1)
        bin_launches.append(e)
    code, st = fr.status()
    if code not in (_abi.GS_OK, _abi.GS_ERR_NUMERIC):
        raise RuntimeError(f"timed binning failed: {_abi.status_string(code)}")

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t0.record(stream)
    for k in range(args.steps):
        step(events[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    code, st = fr.status()
    if code not in (_abi.GS_OK, _abi.GS_ERR_NUMERIC):
        raise RuntimeError(f"timed step failed: {_abi.status_string(code)}")
    total_ms = t0.elapsed_time(t1)
    stage_ms = {s: float(np.mean([events[k][i].elapsed_time(events[k][i + 1]) for k in range(args.steps)]))
                for i, s in enumerate(stages)}
    total_ms = max_over_ranks(total_ms, world, dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(world, args.steps, total_ms)

    # ---- end to end through the public API with host buffers --------------------------------
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, g, gt, fr, dimg, bg, img, T, last, grads, stream, world, dev)

    hbm_peak, peak_kind = load_peaks()
    P = cam.width * cam.height
    sh_floats = 48
    bytes_ = byte_model(gt.n, n_vis, K, segs, P, fr.tiles, sh_floats, fr.layout)
    kernels = {}
    for s in stages:
        kernels[s] = {"ms": round(stage_ms[s], 4), "alg_bytes": int(bytes_[s]),
                      "gbs": round(bytes_[s] / (stage_ms[s] * 1e-3) / 1e9, 1)}
    kernels["bin_sort"]["launches"] = bin_launches
    # Render kernels: the backward walks exactly sum(last) (pixel, splat) pairs and blends
    # `blended` of them; the forward evaluates at least those pairs and blends the same ones.
    flops_fwd = sum_last * FLOPS_EVAL + blended * FLOPS_BLEND_FWD
    flops_bwd = sum_last * FLOPS_EVAL + blended * FLOPS_BLEND_BWD
    kernels["render_forward"]["alg_tflops"] = round(flops_fwd / (stage_ms["render_forward"] * 1e-3) / 1e12, 2)
    kernels["render_backward_tiles"]["alg_tflops"] = round(
        flops_bwd / (stage_ms["render_backward_tiles"] * 1e-3) / 1e12, 2)
    # The roofline is reported for the dominant single kernel; gs_bin_sort is a sequence of
    # ten launches and is reported per stage only.
    single = ["preprocess", "render_forward", "render_backward_tiles", "render_backward_gaussians"]
    dom = max(single, key=lambda s: stage_ms[s])
    traffic = TRAFFIC.get(dom) if args.gaussians == CONFIG3_N else None
    if dom in ("render_forward", "render_backward_tiles"):
        fl = flops_fwd if dom == "render_forward" else flops_bwd
        ach = fl / (stage_ms[dom] * 1e-3) / 1e12
        pk = peaks["fma_tflops"]
        roof = {"kernel": KERNEL_NAMES[dom], "bound": "alu", "achieved": round(ach, 3),
                "peak": pk, "unit": "TFLOP/s", "frac": round(ach / pk, 4),
                "traffic": traffic,
                "peak_kind": f"measured: FP32 FMA microbenchmark (gs_peak_fma, {peaks['blocks']} x 1024 threads, "
                             f"median {peaks['clocks'].get('sm_mhz')} MHz) in this run; nominal "
                             f"{ALU_NOMINAL_TFLOPS:.1f}",
                "units": f"{int(sum_last)} walked (pixel, splat) pairs x {FLOPS_EVAL} + {blended} blended pairs x "
                         f"{FLOPS_BLEND_FWD if dom == 'render_forward' else FLOPS_BLEND_BWD} flops",
                "alg_bytes": int(bytes_[dom]),
                "hbm_frac": round(bytes_[dom] / (stage_ms[dom] * 1e-3) / 1e9 / hbm_peak, 4)}
    else:
        ach = bytes_[dom] / (stage_ms[dom] * 1e-3) / 1e9
        roof = {"kernel": KERNEL_NAMES[dom], "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(ach / hbm_peak, 4), "traffic": traffic,
                "peak_kind": f"{peak_kind} hbm_gbs"}

    # forward-only rendering of the same frame (preprocess + binning + blend), the paper's
    # real-time measure
    render_only = None
    if not args.no_batch:
        for _ in range(3):
            fr.preprocess(gt)
            fr.bin_sort()
            fr.render_forward(bg, img, T, last)
        torch.cuda.synchronize()
        ra, rb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ra.record(stream)
        for _ in range(args.steps):
            fr.preprocess(gt)
            fr.bin_sort()
            fr.render_forward(bg, img, T, last)
        rb.record(stream)
        torch.cuda.synchronize()
        r_ms = ra.elapsed_time(rb) / args.steps
        render_only = {"what": "preprocess + bin_sort + render_forward of the same frame", "ms": round(r_ms, 4),
                       "frames_per_s": round(1e3 / r_ms, 1)}

    # one training iteration (Sec. 5.1): forward, L1 + D-SSIM loss against a synthetic target
    # view, backward, Adam with the activations, on the same scene
    train = None
    if not args.no_batch:
        from paper_2308_04079_gb300.training import GaussianModel, Trainer
        model = GaussianModel.from_numpy(g, device=dev)
        trainer = Trainer(model, bg=bg)
        target = torch.from_numpy(np.random.default_rng(77).random((3, cam.height, cam.width),
                                                                   dtype=np.float32)).to(dev)
        for _ in range(3):
            trainer.step(cam, target)
        torch.cuda.synchronize()
        ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ta.record(stream)
        for _ in range(args.steps):
            out = trainer.step(cam, target)
        tb.record(stream)
        torch.cuda.synchronize()
        codes = trainer.status()
        t_ms = ta.elapsed_time(tb) / args.steps
        train = {"what": "forward + L1/D-SSIM loss (lambda 0.2) + backward + fused activation/Adam of all "
                         "parameters, synthetic target", "ms": round(t_ms, 4),
                 "iterations_per_s": round(1e3 / t_ms, 1), "loss": round(float(out[0].item()), 6),
                 "status": sorted(set(int(c) for c in codes.values()))}
        del trainer, model

    density = variants = None
    if not args.no_batch:
        density = run_density(args, dev, stream, hbm_peak, peak_kind)
        variants = run_variants(args, dev, stream, g, cam, bg, d_dimg, ms_per_step)

    batch = multi = None
    if not args.no_batch and args.gaussians == CONFIG3_N:
        batch = run_batch(args, dev)
        multi = run_multiscene(args, dev)

    cpu = small = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, cam, bg, dimg)
        if args.gaussians == CONFIG3_N:
            small = run_small_configs(dev, stream)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(gt.n, cam, (cfg.tile_w, cfg.tile_h), world),
        "workload_stats": {"sort_mode": args.sort_mode, "visible": n_vis, "instances": K, "segments": segs,
                           "tiles": int(fr.tiles), "mean_list_length": round(K / fr.tiles, 2),
                           "sum_last": int(sum_last), "blended_pairs": blended},
        "alu_peaks": peaks,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "render_only": render_only, "train_step": train, "density_control": density, "variants": variants,
        "batch": batch,
        "multi_scene": multi,
        "small_configs": small,
        "gpu_launches": launches_per_step(fr.layout) * args.steps, "kernels": kernels,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_density(args, dev, stream, hbm_peak, peak_kind):
    """One refinement (Sec. 5.2) of a model of the bench's size: gs_densify over the optimiser
    state of synthetic.density_state (every decision in play), timed with CUDA events; the
    roofline counts the bytes the compaction must move."""
    import torch
    import synthetic as S
    from paper_2308_04079_gb300 import _abi
    from paper_2308_04079_gb300.density import PARAMS, _arrays
    n = args.gaussians
    f, m, v, acc, cnt, mr, z = S.density_state(9000, n)
    up = lambda a: torch.from_numpy(a).to(dev)
    src, sm, sv = ({k: up(d[k]) for k in PARAMS} for d in (f, m, v))
    ta, tc, tm, tz = up(acc), up(cnt), up(mr), up(z)
    del f, m, v, acc, cnt, mr, z
    cap = 2 * n
    out, om, ov = ({k: torch.empty((cap,) + tuple(src[k].shape[1:]), dtype=torch.float32, device=dev)
                    for k in PARAMS} for _ in range(3))
    stats = [torch.empty(cap, dtype=torch.float32, device=dev) for _ in range(3)]
    scales = torch.empty((cap, 3), dtype=torch.float32, device=dev)
    opac = torch.empty(cap, dtype=torch.float32, device=dev)
    result = torch.zeros(2, dtype=torch.int32, device=dev)
    sb = _abi.gs_densify_scratch_size(n)
    scratch = torch.empty(sb + 256, dtype=torch.uint8, device=dev)
    sp = scratch.data_ptr() + (-scratch.data_ptr()) % 256
    cfg = _abi.gs_density_config()
    cfg.grad_threshold, cfg.min_opacity, cfg.split_scale = 2e-4, 0.005, 0.03
    cfg.max_world_scale, cfg.max_screen_radius, cfg.split_factor = 0.3, 20.0, 1.6
    sh_floats = int(src["sh"][0].numel())
    args_ = (cfg, n, sh_floats, _arrays(src), _arrays(sm), _arrays(sv), ta.data_ptr(), tc.data_ptr(), tm.data_ptr(),
             tz.data_ptr(), _arrays(out), _arrays(om), _arrays(ov), stats[0].data_ptr(), stats[1].data_ptr(),
             stats[2].data_ptr(), scales.data_ptr(), opac.data_ptr(), cap, result.data_ptr(), sp, sb,
             stream.cuda_stream)
    for _ in range(3):
        _abi.gs_densify(*args_)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        _abi.gs_densify(*args_)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    rows, flags = (int(x) for x in result.cpu())
    # decisions, from the kernel's own outputs: rows = keep + 2 (clone + split)
    opac_thr = float(np.float32(np.log(0.005 / 0.995)))
    lo = src["logit_opacities"]
    smax = src["log_scales"].max(dim=1).values
    pruned = int(((lo < opac_thr) | (smax > float(np.float32(np.log(0.3)))) | (tm > 20.0)).sum().item())
    dens = (tc > 0) & (ta / torch.where(tc > 0, tc, torch.ones_like(tc)) > float(np.float32(2e-4)))
    keep_mask = ~((lo < opac_thr) | (smax > float(np.float32(np.log(0.3)))) | (tm > 20.0))
    split = int((dens & keep_mask & (smax > float(np.float32(np.log(0.03))))).sum().item())
    row_bytes = 3 * (4 * (3 + 3 + 4 + 1) + 4 * sh_floats)      # value + 2 moments of the 5 tensors
    alg = n * 28 + (n - pruned) * (row_bytes - 16) + split * 24 + rows * (row_bytes + 12 + 16)
    ach = alg / (ms * 1e-3) / 1e9
    return {"what": "gs_densify: prune / clone / split compaction of the parameters and Adam moments "
                    "(Sec. 5.2), synthetic optimiser state", "gaussians": n, "rows_out": rows, "flags": flags,
            "pruned": pruned, "split": split, "ms": round(ms, 4), "algorithmic_bytes": int(alg),
            "achieved_gbs": round(ach, 1), "frac": round(ach / hbm_peak, 4), "peak": hbm_peak,
            "peak_kind": f"{peak_kind} hbm_gbs", "l2": "inputs larger than L2"}


def run_variants(args, dev, stream, g, cam, bg, d_dimg, plain_ms):
    """The ablation variants of Sec. 7.3 on the same frame: Limited-BW (gradients for the 10
    front-most blended splats of each pixel) and isotropic Gaussians (one scale per Gaussian,
    the geometric mean of the three axes), each a whole forward + backward step."""
    import torch
    from paper_2308_04079_gb300 import Frame, GaussianTensors, make_config
    out = {}
    iso_scales = np.exp(np.log(np.asarray(g.scales, np.float64)).mean(axis=1)).astype(np.float32)
    for name, kw in (("limited_bw_n10", dict(grad_limit=10)), ("isotropic", dict(isotropic=True))):
        cfg = make_config(sort_mode=args.sort_mode, **kw)
        gt = GaussianTensors.from_numpy(g, device=dev)
        if kw.get("isotropic"):
            gt = GaussianTensors(gt.means, torch.from_numpy(iso_scales).to(dev), None, gt.opacities, gt.sh,
                                 gt.sh_degree)
        gt = gt.prepared()
        fr = Frame(gt.n, cam, cfg, device=dev)
        fr.ensure_binned(gt)
        fr = Frame(gt.n, cam, cfg, capacity=int(fr.last_status.num_instances * 1.15) + 4096, device=dev)
        img, T, last = fr.outputs()
        grads = fr.new_grads(gt)

        def step():
            fr.preprocess(gt)
            fr.bin_sort()
            fr.render_forward(bg, img, T, last)
            fr.render_backward(gt, bg, d_dimg, T, last, grads)
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        code, st = fr.status()
        ms = a.elapsed_time(b) / args.steps
        out[name] = {"ms": round(ms, 4), "frames_per_s": round(1e3 / ms, 1), "vs_full_method": round(plain_ms / ms, 3),
                     "instances": int(st.num_instances), "status": int(code)}
        del fr, img, T, last, grads, gt
    out["what"] = ("whole forward + backward step of the Sec. 7.3 ablations on the same frame; vs_full_method = "
                   "the full method's ms / the variant's ms")
    return out


def frame_stats(frames, lasts=None, backward=True):
    """Workload figures of a config, summed over its frames: visible Gaussians, instances K,
    segment records, tiles, the mean tile list length K / tiles and, when given, the walked
    (pixel, splat) pairs (the sum of every pixel's last position) and the blended pairs of the
    last backward pass."""
    import torch
    vis = K = segs = tiles = blended = 0
    for f in frames:
        _, st = f.status()
        vis += int(st.num_visible)
        K += int(st.num_instances)
        segs += int(st.num_segments)
        blended += int(st.blended_pairs)
        tiles += int(f.tiles)
    out = {"frames": len(frames), "visible": vis, "instances": K, "segments": segs, "tiles": tiles,
           "mean_list_length": round(K / max(tiles, 1), 2)}
    if lasts is not None:
        out["sum_last"] = int(sum(float(x.to(torch.float64).sum().item()) for x in lasts))
    if backward:
        out["blended_pairs"] = blended
    return out


def run_batch(args, dev):
    """Config 4: one 1M-Gaussian scene (config-3 distribution), 16 views of uneven size,
    forward+backward with the gradients summed over the views -- as one batch (one launch per
    kernel for all views) and as the plain per-view loop on the same frames."""
    import torch
    import synthetic as S
    from paper_2308_04079_gb300 import Frame, FrameBatch, GaussianTensors, make_config
    g, cams, bg, dimgs = S.config4(n=args.batch_gaussians, views=args.batch_views)
    bg = tuple(float(x) for x in bg)
    gt = GaussianTensors.from_numpy(g, device=dev).prepared()
    d = [torch.from_numpy(x).to(dev) for x in dimgs]
    cfg = make_config()
    frames = [Frame(gt.n, cam, cfg, device=dev) for cam in cams]
    batch = FrameBatch(frames, [gt] * len(frames))
    batch.ensure_binned()
    frames = [Frame(gt.n, cam, cfg, capacity=int(f.last_status.num_instances * 1.15) + 4096, device=dev)
              for cam, f in zip(cams, frames)]
    batch = FrameBatch(frames, [gt] * len(frames))
    outs = batch.outputs()
    grads = frames[0].new_grads(gt)
    stream = torch.cuda.current_stream()

    def batched():
        batch.preprocess()
        batch.bin_sort()
        batch.render_forward(bg, outs)
        batch.render_backward(bg, d, outs, [grads] * len(frames))

    def per_view():
        for v, f in enumerate(frames):
            f.preprocess(gt)
            f.bin_sort()
            f.render_forward(bg, *outs[v])
            f.render_backward(gt, bg, d[v], outs[v][1], outs[v][2], grads, accumulate=v > 0)

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    steps = max(3, min(args.steps, 10))
    ms_loop = timed(per_view, steps)
    img_loop = [o[0].clone() for o in outs]
    ms_batch = timed(batched, steps)
    same = all(torch.equal(o[0], x) for o, x in zip(outs, img_loop))
    for f in frames:
        code, _ = f.status()
        if code not in (0, 5):
            raise RuntimeError(f"batched frame failed with status {code}")
    stats = frame_stats(frames, [o[2] for o in outs])
    sizes = sorted({(c.width, c.height) for c in cams})
    return {"workload": f"one scene of {gt.n} Gaussians (config-3 distribution), {len(frames)} views of uneven size "
                        f"({', '.join(f'{w}x{h}' for w, h in sizes)}), forward+backward, gradients summed over views",
            "views": len(frames), "batched_ms": round(ms_batch, 4), "per_view_ms": round(ms_loop, 4),
            "speedup": round(ms_loop / ms_batch, 3), "views_per_s": round(len(frames) / (ms_batch * 1e-3), 1),
            "images_identical": bool(same), "steps": steps, "workload_stats": stats}


def run_multiscene(args, dev):
    """Config 5: 8 independent scenes (log-uniform 50k-2M Gaussians, SH degree 3), 4 views each
    at mixed resolutions, forward+backward of all 32 frames captured in one CUDA graph at the
    autotuned tile shape and batch depth; against the plain per-view loop at the same config."""
    import torch
    import synthetic as S
    from paper_2308_04079_gb300 import GaussianTensors
    from paper_2308_04079_gb300.batching import Scene, SceneBatch, autotune
    raw, bg = S.config5()
    bg = tuple(float(x) for x in bg)
    scenes = [Scene(GaussianTensors.from_numpy(g, device=dev).prepared(), cams,
                    [torch.from_numpy(d).to(dev) for d in dl]) for g, cams, dl in raw]
    cfg, table = autotune(scenes, bg, steps=3)
    sb = SceneBatch(scenes, bg, cfg)
    sb.capture()
    steps = max(3, min(args.steps, 10))
    ms_graph = sb.time_replay(steps)
    sb.check()
    stream = torch.cuda.current_stream()

    def plain():
        for f, o, d, gr, g in zip(sb.frames, sb.outs, sb.dl, sb.view_grads, sb.batch.gaussians):
            f.preprocess(g)
            f.bin_sort()
            f.render_forward(sb.bg, *o)
            f.render_backward(g, sb.bg, d, o[1], o[2], gr, accumulate=id(gr) in plain.done)
            plain.done.add(id(gr))

    def run_plain():
        plain.done = set()
        plain()

    for _ in range(3):
        run_plain()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        run_plain()
    b.record(stream)
    torch.cuda.synchronize()
    ms_plain = a.elapsed_time(b) / steps
    stats = frame_stats(sb.frames, [o[2] for o in sb.outs])
    return {"workload": f"{len(scenes)} scenes of {', '.join(str(s.gaussians.n) for s in scenes)} Gaussians, "
                        f"{len(sb.frames)} frames at mixed resolutions, forward+backward, one CUDA graph",
            "tile": f"{cfg.tile_w}x{cfg.tile_h}", "batch_depth": int(cfg.batch_depth),
            "autotune": [{"tile": f"{t[0]}x{t[1]}", "batch_depth": d, "ms": round(ms, 4)} for t, d, ms in table],
            "graph_ms": round(ms_graph, 4), "plain_ms": round(ms_plain, 4), "speedup": round(ms_plain / ms_graph, 3),
            "frames_per_s": round(len(sb.frames) / (ms_graph * 1e-3), 1), "steps": steps, "workload_stats": stats}


def run_e2e(args, g, gt, fr, dimg, bg, img, T, last, grads, stream, world, dev):
    """Same metric through the public API with pinned host buffers: every step copies the
    Gaussian parameters and dL/dimage in, runs the four stages, and copies the image and all
    gradients out.  The inputs of a step sit in one pinned host slab and one device slab (the
    tensors the stages read are views into it), the outputs likewise, so each step moves its
    bytes with one host-to-device and one device-to-host copy.  Steps are pipelined two deep on
    three streams (copy in, compute, copy out) with double-buffered slabs, so the copies of
    neighbouring steps overlap the compute of the current one; every step still moves all of
    its bytes.  The copies' own rates are measured with events on the copy streams."""
    import torch
    from paper_2308_04079_gb300 import GaussianTensors

    def layout(shapes):
        """Offsets (in floats, 16-byte aligned) of tensors of the given shapes in one slab."""
        offs, o = [], 0
        for sh in shapes:
            offs.append(o)
            o += (int(np.prod(sh)) + 3) // 4 * 4
        return offs, o

    names = ("means", "scales", "quats", "opacities", "sh")
    in_shapes = [tuple(getattr(gt, k).shape) for k in names] + [tuple(dimg.shape)]
    in_offs, in_len = layout(in_shapes)
    out_keys = ["image"] + list(grads.keys())
    out_shapes = [tuple(img.shape)] + [tuple(v.shape) for v in grads.values()]
    out_offs, out_len = layout(out_shapes)

    def views(slab, offs, shapes):
        return [slab[o:o + int(np.prod(sh))].view(sh) for o, sh in zip(offs, shapes)]

    host_in = torch.empty(in_len, dtype=torch.float32).pin_memory()
    for v, a in zip(views(host_in, in_offs, in_shapes), [getattr(g, k) for k in names] + [dimg]):
        v.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)))
    host_out = [torch.empty(out_len, dtype=torch.float32).pin_memory() for _ in range(2)]
    dev_in = [torch.empty(in_len, dtype=torch.float32, device=dev) for _ in range(2)]
    dev_out = [torch.empty(out_len, dtype=torch.float32, device=dev) for _ in range(2)]
    ins, outs = [], []
    for b in range(2):
        iv = views(dev_in[b], in_offs, in_shapes)
        ins.append((GaussianTensors(*iv[:5], gt.sh_degree), iv[5]))
        ov = dict(zip(out_keys, views(dev_out[b], out_offs, out_shapes)))
        o_img = ov.pop("image")
        outs.append((o_img, torch.empty_like(T), torch.empty_like(last), ov))
    h2d = in_len * 4
    d2h = out_len * 4
    steps = max(3, min(args.steps, 10))
    s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    tev = lambda: torch.cuda.Event(enable_timing=True)
    in_ready, used, done, drained = [ev(), ev()], [ev(), ev()], [ev(), ev()], [ev(), ev()]
    copy_ev = [(tev(), tev(), tev(), tev()) for _ in range(steps + 2)]
    for e in used + drained:            # both buffer sets start free
        e.record(stream)

    def step(k):
        b = k % 2
        g_dev, d_dev = ins[b]
        o_img, o_T, o_last, o_grads = outs[b]
        c0, c1, c2, c3 = copy_ev[k]
        with torch.cuda.stream(s_in):
            s_in.wait_event(used[b])           # the compute two steps back has read this set
            c0.record(s_in)
            dev_in[b].copy_(host_in, non_blocking=True)
            c1.record(s_in)
            in_ready[b].record(s_in)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(in_ready[b])
            s_comp.wait_event(drained[b])      # the outputs two steps back are copied out
            fr.preprocess(g_dev)
            fr.bin_sort()
            fr.render_forward(bg, o_img, o_T, o_last)
            fr.render_backward(g_dev, bg, d_dev, o_T, o_last, o_grads)
            used[b].record(s_comp)
            done[b].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(done[b])
            c2.record(s_out)
            host_out[b].copy_(dev_out[b], non_blocking=True)
            c3.record(s_out)
            drained[b].record(s_out)

    for k in range(2):
        step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for q in (s_in, s_comp, s_out):
        q.wait_event(a)
    for k in range(steps):
        step(k + 2)
    for e in drained:
        stream.wait_event(e)
    z.record(stream)
    torch.cuda.synchronize()
    val = job_rate(world, steps, max_over_ranks(a.elapsed_time(z), world, dev))
    t_in = float(np.median([copy_ev[k + 2][0].elapsed_time(copy_ev[k + 2][1]) for k in range(steps)]))
    t_out = float(np.median([copy_ev[k + 2][2].elapsed_time(copy_ev[k + 2][3]) for k in range(steps)]))
    # the same frame's outputs came back intact
    o = host_out[(steps + 1) % 2]
    ok = bool(torch.equal(o[out_offs[0]:out_offs[0] + img.numel()].view(img.shape), img.cpu()))
    return {"value": round(val, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": steps, "h2d_gbs": round(h2d / (t_in * 1e-3) / 1e9, 1),
            "d2h_gbs": round(d2h / (t_out * 1e-3) / 1e9, 1), "image_matches_device_run": ok,
            "pipelining": "one pinned slab per direction per step (one H2D and one D2H copy); 2 steps in flight: "
                          "H2D, compute and D2H on separate streams"}


# ------------------------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ------------------------------------------------------------------------------------------
def oracle_frame(g, cam, bg, dimg) -> float:
    """Seconds the FP64 oracle takes for one whole frame: forward (image, T, last) and
    backward (every gradient) of all tiles, on all host cores.  The backward runs without the
    tests' allowances (the flipped-decision and conditioning terms), which are test machinery,
    not the method."""
    import oracle
    t = time.perf_counter()
    oracle.render_forward(g, cam, bg)
    oracle.render_backward(g, cam, dimg, bg, allowance=False)
    return time.perf_counter() - t


def _f64_gaussians(g):
    import synthetic as S
    return S.Gaussians(*(np.asarray(a, np.float64) for a in (g.means, g.scales, g.quats, g.opacities, g.sh)),
                       g.sh_degree)


def cpu_baseline(g, cam, bg, dimg):
    import oracle
    s = oracle_frame(_f64_gaussians(g), cam, bg, dimg)
    tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    sample = (f"FP64 oracle: one whole frame, preprocess of all {g.n} Gaussians + forward and backward of "
              f"all {tiles} 16x16 tiles ({s:.1f} s)")
    return {"value": round(1.0 / s, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": sample}


def run_small_configs(dev, stream):
    """Configs 1 (1k Gaussians, 128x128, forward only) and 2 (200k Gaussians, 1080p, forward +
    backward): the GPU's time per frame through the same calls as the main step (CUDA events,
    median of 20 after 5 warm-ups) beside the FP64 oracle's time for the same frame on all host
    cores."""
    import torch
    import oracle
    import synthetic as S
    from paper_2308_04079_gb300 import Frame, GaussianTensors, make_config
    out = {}
    for name, fn in (("config1", S.config1), ("config2", S.config2)):
        res = fn()
        g, cam, bg = res[0], res[1], tuple(float(x) for x in res[2])
        dimg = res[3] if len(res) > 3 else None
        gt = GaussianTensors.from_numpy(g, device=dev).prepared()
        fr = Frame(gt.n, cam, make_config(), device=dev)
        fr.ensure_binned(gt)
        img, T, last = fr.outputs()
        d = torch.from_numpy(dimg).to(dev) if dimg is not None else None
        grads = fr.new_grads(gt)

        def frame():
            fr.preprocess(gt)
            fr.bin_sort()
            fr.render_forward(bg, img, T, last)
            if d is not None:
                fr.render_backward(gt, bg, d, T, last, grads)

        for _ in range(5):
            frame()
        torch.cuda.synchronize()
        times = []
        for _ in range(20):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            frame()
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        g64 = _f64_gaussians(g)
        t0 = time.perf_counter()
        if d is None:
            oracle.render_forward(g64, cam, bg)
        else:
            oracle.render_backward(g64, cam, dimg, bg, allowance=False)
            oracle.render_forward(g64, cam, bg)
        t_orc = time.perf_counter() - t0
        out[name] = {"what": "forward" if d is None else "forward + backward", "gaussians": gt.n,
                     "size": f"{cam.width}x{cam.height}", "gpu_ms": round(float(np.median(times)), 4),
                     "oracle_s": round(t_orc, 3), "oracle_cores": oracle.num_threads(),
                     "workload_stats": frame_stats([fr], [last], backward=d is not None)}
    return out


def run_reference(args, rank, world):
    """The FP64 oracle as it stands on the host cores, on the same frame: each step is one whole
    frame, forward and backward (the same work as one step of our arm)."""
    if rank != 0:
        return
    import oracle
    import synthetic as S
    g, cam, bg, dimg = S.config3()
    bg = tuple(float(x) for x in bg)
    g64 = _f64_gaussians(g)
    for _ in range(args.warmup):
        oracle_frame(g64, cam, bg, dimg)
    t = time.perf_counter()
    per_step = [oracle_frame(g64, cam, bg, dimg) for _ in range(args.steps)]
    wall = time.perf_counter() - t
    ms_per_step = wall / args.steps * 1e3
    value = args.steps / wall
    cores = oracle.num_threads()
    tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    sample = (f"each step one whole frame: FP64 oracle preprocess of all {g.n} Gaussians + forward and backward "
              f"of all {tiles} 16x16 tiles (per step {min(per_step):.1f}-{max(per_step):.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(g.n, cam, (16, 16), world),
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sort-mode", choices=["two_phase", "key64"], default="two_phase")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched multi-view and multi-scene comparisons")
    ap.add_argument("--batch-gaussians", type=int, default=1_000_000)
    ap.add_argument("--batch-views", type=int, default=16)
    ap.add_argument("--gaussians", type=int, default=CONFIG3_N,
                    help="Gaussians of the config-3 scene (smaller counts for profiling captures)")
    ap.add_argument("--density-only", action="store_true",
                    help="time one density-control refinement (gs_densify) of --gaussians Gaussians only")
    ap.add_argument("--peaks-only", action="store_true",
                    help="measure and print the FP32 FMA and 2^x peaks of GPU 0 only")
    args = ap.parse_args()
    if args.peaks_only:
        import torch
        from paper_2308_04079_gb300 import build as gbuild
        torch.cuda.set_device(0)
        if gbuild.needs_build():
            gbuild.build()
        print(json.dumps(measure_alu_peaks(torch.device("cuda", 0), seconds=2.0)), flush=True)
        return
    if args.density_only:
        import torch
        from paper_2308_04079_gb300 import build as gbuild
        torch.cuda.set_device(0)
        if gbuild.needs_build():
            gbuild.build()
        hbm_peak, peak_kind = load_peaks()
        print(json.dumps(run_density(args, torch.device("cuda", 0), torch.cuda.current_stream(), hbm_peak,
                                     peak_kind)), flush=True)
        return
    rank, world, local_rank = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        # The CPU oracle runs on rank 0 only; other ranks exit without work.
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
