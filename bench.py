"""Benchmark: LiDAR rays/s on the 128-channel, 2048-azimuth (262,144 beams)
sensor over the 1,036,288-triangle terrain + objects scene.

One step = one pass of the whole per-beam path for one frame: ray generation,
closest-hit traversal, surface attributes, incidence angle, reflectance lerp,
Philox range noise, cut-offs, intensity and the ordered compaction of the
kept returns into a point cloud.  The BVH is built once per scene (timed
separately, reported as build_ms).  L2 is flushed (256 MiB write) before every
timed step.  The launch configuration and ray schedule come from the
autotuner; the cost schedule is measured on a pose 1.1 m away from the timed
one (as the previous frame of a moving sensor would be).

Also reported (extra keys): the 8-sensor x 64-frame batch replayed as one
CUDA graph, forward + adjoint of the 16-frame differentiation workload next to
the plain single-frame forward, and the ~10.7M-triangle city with 7 sub-rays.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(brute force, OpenMP) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LiDAR rays/sec (128-ch, 1M-tri scene) & roofline %; fwd+bwd vs plain fwd ms"
UNIT = "rays/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK_GBS = 6800.0
# The launch the headline kernel's ncu captures ran (k_cast<0, 2, 2>)
HEADLINE_LAUNCH = {"traversal": (2,), "block_threads": (256,), "blocks_per_sm": (2,)}
# The launches the end-to-end (streaming) loop chooses among: the 4-wide walk
# at 256 threads per block, 2 or 3 blocks per SM (128 or 85 registers)
STREAM_LAUNCH = {"traversal": (2,), "block_threads": (256,), "blocks_per_sm": (2, 3)}
# The hierarchies the benchmark walks: PLOC plus rounds of treelet
# restructuring, with the builders' area measure weighting the boxes' top and
# bottom faces (normal to z) less than their sides — the choices that cast
# fastest on a GB300 among the round counts, weights, PLOC radii and triangle
# costs measured (one frame each, L2 flushed)
CFG1_TREE = {"treelet_rounds": 2, "area_weight": (1.0, 1.0, 0.23)}
CITY_TREE = {"treelet_rounds": 8, "area_weight": (1.0, 1.0, 0.35)}


def tree_name(tree):
    return (f"PLOC + {tree['treelet_rounds']} treelet rounds, face weights "
            f"{'/'.join(f'{v:g}' for v in tree['area_weight'])} (x/y/z), collapsed 4-wide")


POINT_BYTES = 12 + 4 + 4 + 12 + 2 + 4 + 4 + 4   # xyz, range, intensity, normal, material, instance, beam, frame


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the cast kernel as the roofline times it (cfg1 frame, dense valid flags out,
# L2 flushed before the launch), from one ncu capture, with the digest of the
# kernel sources the capture ran.  Reported only while the sources still match.
NCU_TRAFFIC = {"sources": "43cc999e0fe54cea", "tree": dict(treelet_rounds=2, area_weight=(1.0, 1.0, 0.23)),
               "bytes": 9_744_640, "l2_bytes": 3_380_907 * 32,
               "l1_global_load_bytes": 6_591_193 * 32}   # profiles/k_cast_cfg1_ncu_full.md
# Binding-unit fractions of the same capture (ncu --set full of one launch):
# L1/TEX throughput, issue-active and SM-active shares.
NCU_UNITS = {"l1tex_throughput_pct": 41.1, "issue_active_pct": 43.4, "sm_active_pct": 71.0}
# FP32 work of one launch of the cast kernel from ncu's SASS instruction
# counters (sm__sass_thread_inst_executed_op_{ffma,fadd,fmul,ffma2,fadd2,fmul2,
# fp32}_pred_on), FLOPs = 2 ffma + fadd + fmul + 4 ffma2 + 2 fadd2 + 2 fmul2 +
# the remaining FP32 instructions (min/max, compares) once each.
NCU_FP32 = {"sources": "43cc999e0fe54cea", "tree": dict(treelet_rounds=2, area_weight=(1.0, 1.0, 0.23)),
            "fp32_flops": 497_878_528, "fp32_ops": 476_442_679,
            "counters": {"ffma": 21_435_849, "fadd": 10_460_945, "fmul": 33_010_988, "ffma2": 0,
                         "fadd2": 68_563_704, "fmul2": 68_563_704, "fp32_all": 339_315_271}}
# profiles/k_cast_cfg1_fp32_counts.md
# Binding-unit fractions of one city frame launch (ncu --set full,
# profiles/k_cast_city_ncu_full.md), with the sources and tree it ran
NCU_CITY_UNITS = {"sources": "43cc999e0fe54cea", "tree": dict(treelet_rounds=8, area_weight=(1.0, 1.0, 0.35)),
                  "kernel": "k_cast<0, 4, 2>",
                  "issue_active_pct": 74.8, "l1tex_throughput_pct": 62.9, "fma_pipe_pct": 42.7, "alu_pipe_pct": 53.5}
KERNEL_SOURCES = ("cast.cu", "shade.cuh", "trace.cuh", "common.cuh", "philox.cuh")
# DRAM traffic (read + write) of one launch of the one-pass adjoint on the
# 16-frame tape, from one ncu capture (profiles/k_adj_cfg3_ncu_full.md),
# reported while adjoint.cu still has the captured digest
ADJ_TRAFFIC = {"sources": "0d4c79dc0d5a7f66", "bytes": 67_204_352 + 2_014_464}


def kernel_digest():
    """Digest of the sources that make up the cast kernel (of common.cuh only
    the device-side layout above its host launcher declarations)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2208_10295_gb300", "csrc", f), "rb") as fh:
            data = fh.read()
        if f == "common.cuh":
            data = data[:data.find(b"// ------------------------------------------------------------------ kernel launchers")]
        h.update(data)
    return h.hexdigest()[:16]


def kernel_name(cfg):
    """The cast kernel instantiation a launch configuration runs: k_cast<0,
    register variant, traversal>, the variant from the requested residency
    (threads x blocks per SM <= 512: 128 registers, <= 768: 85, else 64)."""
    threads = cfg["block_threads"] * cfg["blocks_per_sm"]
    variant = 2 if threads <= 512 else (3 if threads <= 768 else 4)
    return f"k_cast<0, {variant}, {cfg['traversal']}>"


def adjoint_digest():
    import hashlib
    with open(os.path.join(ROOT, "paper_2208_10295_gb300", "csrc", "adjoint.cu"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def build_with_tree(L, w, tree):
    """w's scene as a PLOC hierarchy with the options in `tree`; the
    context's build options are restored afterwards."""
    opts = L.build_options()
    L.set_build_options(method=1, ploc_radius=opts["ploc_radius"], **tree)
    try:
        return L.build_scene(w.scene.verts, w.scene.tris, w.scene.mat, w.scene.inst)
    finally:
        L.set_build_options(**opts)


def build_cfg1(L, w):
    """The 1.04M-triangle scene (cfg1, and the batches and tapes cast in it)."""
    return build_with_tree(L, w, CFG1_TREE)


def build_city(L, w4):
    """The 10.7M-triangle city (cfg4)."""
    return build_with_tree(L, w4, CITY_TREE)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": HBM_FALLBACK_GBS, "sm_max_mhz": 2070.0}, "fallback"


def shard_frames(n_frames_total: int, rank: int, world: int):
    """Contiguous block of frame indices owned by `rank` (weak scaling: each
    rank gets the same number of frames)."""
    per = n_frames_total // world
    return list(range(rank * per, (rank + 1) * per))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"lidar_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measure_fp32_peak(L, gpu_index, seconds=1.0):
    """FP32 FMA rate measured on this GPU (the library's probe kernel: every SM
    running independent fused multiply-add chains), repeated for about
    `seconds` while nvidia-smi samples the SM clock; the best rate and the
    median clock it ran at."""
    best = None
    with ClockSampler(gpu_index) as clk:
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end or best is None:
            r = L.measure_fp32_rate(1 << 24)
            if best is None or r["flops_per_s"] > best["flops_per_s"]:
                best = r
    c = clk.summary() or {}
    return {"tflops": best["flops_per_s"] / 1e12, "probe_kernel_ms": best["kernel_ms"],
            "packed_pairs": best["packed"], "sm_mhz": c.get("sm_mhz"), "clock_reasons": c.get("reasons")}


def event_time(torch, stream, fn, flush=None, reps=10, warm=2):
    ts = []
    for i in range(reps + warm):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        if i >= warm:
            ts.append(a.elapsed_time(b))
    return statistics.mean(ts)


def run_ours(args, rank, world, local_rank):
    import torch

    import synth
    from paper_2208_10295_gb300 import Lidar
    from paper_2208_10295_gb300.build import build as build_lib
    from paper_2208_10295_gb300.tune import apply as apply_cfg
    from paper_2208_10295_gb300.tune import autotune

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    build_lib()
    dev = torch.device("cuda", local_rank)
    w = synth.cfg1()
    frames = w.frames.copy()
    if world > 1:
        # weak scaling: every rank casts its own frame of the trajectory, no data-path collective
        w3 = synth.cfg3(n_frames=world)
        frames = w3.frames[shard_frames(world, rank, world)].copy()
    L = Lidar(local_rank)
    stream = L.stream
    scene = build_cfg1(L, w)
    L.set_sensor(0, w.sensors[0])
    table = L.build_tables(torch.tensor(w.params, device=dev))
    L.set_materials(table)
    near = frames.copy()
    near[0]["pose"][3] += 1.0
    near[0]["pose"][7] += 0.5
    # the headline's kernel is the one the ncu captures describe: the 4-wide
    # walk at 256 threads x 2 blocks per SM (the 8-wide walk and other shapes
    # measure within a few per cent of it on this tree and would make the
    # captured traffic and unit fractions another kernel's); ray order,
    # schedule and the fused scatter are tuned
    tuned_cfg, tuned_ms = autotune(L, scene, frames, w.seed, schedule_frames=near, use_cache=not args.retune,
                                   points=True, restrict=HEADLINE_LAUNCH)
    n_beams = L.total_beams(frames)
    build_ms = scene.info()["build_ms"]
    pts = L.alloc_points(n_beams)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        L.cast_into(scene, frames, w.seed, None, pts)

    if args.raster_only:
        # the raster-and-resample path alone on the cfg1 frame (profiling runs): 6 cameras, W = 1024
        ras = L.alloc_beams(n_beams, ("valid", "tri", "t"))
        r_ms = event_time(torch, stream, lambda: L.raster_cast_into(scene, frames, w.seed, ras, width=1024,
                                                                    n_cameras=6), flush,
                          reps=args.steps, warm=args.warmup)
        if L.sync_status() != 0:
            raise RuntimeError("device status")
        return {"kernel": "k_raster_tris + k_big_scan + k_raster_big + k_gbuffer + k_resample", "ms": r_ms,
                "width": 1024, "n_cameras": 6, "calls": args.warmup + args.steps} if rank == 0 else None

    if args.city_only:
        # one frame of the city (7 sub-rays per beam) cast to dense valid flags (profiling runs)
        w4 = synth.cfg4()
        scene4 = build_city(L, w4)
        L.set_sensor(0, w4.sensors[0])
        L.set_materials(L.build_tables(torch.tensor(w4.params, device=dev)))
        cfg4, _ = autotune(L, scene4, w4.frames[:4], w4.seed, schedule_frames=w4.frames[:1],
                           use_cache=not args.retune, points=True)
        fr4 = w4.frames[1:2]
        d4 = L.alloc_beams(L.total_beams(fr4), ("valid",))
        c_ms = event_time(torch, stream, lambda: L.cast_into(scene4, fr4, w4.seed, d4), flush,
                          reps=args.steps, warm=args.warmup)
        if L.sync_status() != 0:
            raise RuntimeError("device status")
        return {"kernel": "k_cast", "kernel_ms": c_ms, "launches": args.warmup + args.steps, "launch": cfg4,
                "subrays": L.total_beams(fr4) * 7} if rank == 0 else None

    if args.adjoint_only:
        # the cfg3 fused-MSE backward alone (profiling runs)
        d3 = cfg3_adjoint(torch, L, scene, use_cache=not args.retune)
        d3["fwd"]()
        # the fused-MSE backward call alone: one launch of the one-pass kernel each
        kernel_ms = event_time(torch, stream, d3["bwd_kernel"], flush, reps=args.steps, warm=args.warmup)
        if L.sync_status() != 0:
            raise RuntimeError("device status")
        return {"kernel": "k_adj_onepass", "kernel_ms": kernel_ms, "sources": adjoint_digest(),
                "beams": d3["n"], "launches": args.warmup + args.steps,
                "loss": float(d3["loss"].item())} if rank == 0 else None

    if args.kernel_only:
        # the roofline's kernel alone (profiling runs): cast to dense valid flags
        dense = L.alloc_beams(n_beams, ("valid",))
        kernel_ms = event_time(torch, stream, lambda: L.cast_into(scene, frames, w.seed, dense), flush,
                               reps=args.steps, warm=args.warmup)
        if L.sync_status() != 0:
            raise RuntimeError("device status")
        return {"kernel": "k_cast", "kernel_ms": kernel_ms, "launches": args.warmup + args.steps,
                "launch": tuned_cfg, "sources": kernel_digest()} if rank == 0 else None

    # ---- whole-step timing (cast + compaction), L2 flushed before each step
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        # keep the GPU busy while nvidia-smi starts, so every sample is under load
        t_end = time.perf_counter() + 0.6
        while time.perf_counter() < t_end:
            flush.zero_()
            step()
            torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    st = L.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st}")
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    n_points = int(pts["count"].item())
    # kernels of this library per step: the cast, plus the scatter unless it runs inside the cast
    launches_per_step = 1 if L.launch_config()["fused_scatter"] else 2

    # ---- dominant kernel alone (the cast kernel, dense valid flags out)
    dense = L.alloc_beams(n_beams, ("valid",))
    kernel_ms = event_time(torch, stream, lambda: L.cast_into(scene, frames, w.seed, dense), flush,
                           reps=min(args.steps, 200), warm=3)

    # ---- end to end through host buffers: pose in, point cloud out.  Steps are
    # pipelined: step i's cast (its frame record copied in from pinned memory by
    # the call) is queued while step i-2's point cloud is copied out on a copy
    # stream into pinned host buffers, so two casts are queued ahead of the
    # host's wait for a count and consecutive casts overlap on the GPU.  Four
    # device point buffers rotate: a cast never writes a buffer whose copies
    # have not finished.
    # the launch is tuned for this regime (back-to-back casts, no flush)
    stream_cfg, _ = autotune(L, scene, frames, w.seed, schedule_frames=near, use_cache=not args.retune,
                             points=True, streaming=True, restrict=STREAM_LAUNCH)
    n_buf = 4
    lag = 2
    pbuf = [pts] + [L.alloc_points(n_beams) for _ in range(n_buf - 1)]
    host = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in pts.items()} for _ in range(n_buf)]
    copy_stream = torch.cuda.Stream(device=dev)
    cast_done = [torch.cuda.Event() for _ in range(n_buf)]
    copy_done = [torch.cuda.Event() for _ in range(n_buf)]
    count_ready = torch.cuda.Event()
    n_e2e = min(args.steps, 1000)

    def drain(i):
        """Copies step i's point cloud to the host (count first, then its points)."""
        b = i % n_buf
        copy_stream.wait_event(cast_done[b])
        with torch.cuda.stream(copy_stream):
            host[b]["count"].copy_(pbuf[b]["count"], non_blocking=True)
            count_ready.record(copy_stream)
            count_ready.synchronize()
            c = int(host[b]["count"][0])
            # every field's first c points in one native call (the library's download entry point)
            L.download_points(pbuf[b], host[b], min(c, n_beams), stream=copy_stream)
            copy_done[b].record(copy_stream)
        return c

    bo_total = 0
    for rep in range(2):   # first pass warms up, second is timed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        total_pts = 0
        for i in range(n_e2e + lag):
            if i < n_e2e:
                b = i % n_buf
                # buffer b's previous copy-out is done (waited for on the host, so that
                # consecutive casts follow each other on the stream and may overlap)
                copy_done[b].synchronize()
                L.cast_into(scene, frames, w.seed, None, pbuf[b])
                cast_done[b].record(stream)
            if i >= lag:
                total_pts += drain(i - lag)
        copy_stream.synchronize()
        e2e_s = time.perf_counter() - t0
        bo_total = n_e2e * 8 + total_pts * POINT_BYTES
    e2e_step_ms = e2e_s / n_e2e * 1e3
    del pbuf[1:]
    apply_cfg(L, scene, tuned_cfg, near, w.seed)

    # ---- algorithmic work of one launch (instrumented run of the same kernel)
    counters = L.count_work(scene, frames, w.seed)
    fp32_peak = measure_fp32_peak(L, local_rank) if rank == 0 else None
    # ---- dense records of the timed frame for the parity check against the oracle's sample
    parity_dense = None
    if rank == 0 and world == 1 and not args.no_cpu:
        pf = ("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst")
        pd = L.alloc_beams(n_beams, pf)
        L.cast_into(scene, frames, w.seed, pd)
        if L.sync_status() != 0:
            raise RuntimeError("device status")
        parity_dense = {k: v.cpu().numpy() for k, v in pd.items()}
        del pd

    extras = {}
    if not args.no_extras and world == 1:
        extras = run_extras(args, torch, L, scene, w, table, flush, stream, step, tuned_cfg)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return None
    peaks, peaks_src = load_peaks()
    clocks = clk.summary()
    value = n_beams * args.steps * world / (total_ms / 1e3)
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    visit_bytes = counters["node_visits"] * counters["node_bytes"] + counters["tri_tests"] * 48 + counters["io_bytes"]
    uniq_bytes = counters["unique_node_bytes"] + counters["unique_tri_bytes"] + counters["io_bytes"]
    achieved = visit_bytes / (kernel_ms / 1e3) / 1e9
    captured_launch = all(tuned_cfg.get(k) in v for k, v in HEADLINE_LAUNCH.items())
    same_kernel = (NCU_TRAFFIC["sources"] == kernel_digest() and NCU_TRAFFIC["tree"] == CFG1_TREE and
                   captured_launch)
    traffic = NCU_TRAFFIC["bytes"] if same_kernel else None
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1455.0)
    # FP32 ops per child box of a fetched node: 6 slab subtracts + 6 multiplies, 3 max (entry, with t_eps),
    # 2 min (exit), the far-scale multiply, the min with the best hit and the compare = 20; a node holds
    # node_bytes / 32 children (2, 4 or 8); 40 per watertight triangle test
    flops = counters["node_visits"] * (counters["node_bytes"] // 32) * 20 + counters["tri_tests"] * 40
    alu_tf = flops / (kernel_ms / 1e3) / 1e12
    # the measured FP32 rate, scaled from the probe's clock to the clock the cast ran at
    fp_probe = fp32_peak
    fp_peak = fp_probe["tflops"] * (sm_mhz / fp_probe["sm_mhz"] if fp_probe.get("sm_mhz") else 1.0)
    ncu_ok = NCU_FP32["sources"] == kernel_digest() and NCU_FP32["tree"] == CFG1_TREE and captured_launch
    ncu_fp32_tf = NCU_FP32["fp32_flops"] / (kernel_ms / 1e3) / 1e12 if ncu_ok else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "cfg1: 128-ch x 2048 az (262,144 beams) over the 1,036,288-tri terrain+objects "
                               "scene, one frame per step incl. ordered compaction",
                   "beams_per_step_per_gpu": n_beams, "tris": int(w.scene.n_tris),
                   "l2": "flushed (256 MiB write) before every timed step", "build_ms": build_ms,
                   "tree": tree_name(CFG1_TREE),
                   "points_per_step": n_points, "launch": tuned_cfg},
        "gpu_launches": launches_per_step * args.steps,
        "e2e": {"value": n_beams / (e2e_step_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": 56,
                "d2h_bytes_per_step": bo_total / n_e2e, "steps": n_e2e,
                "how": "host wall clock over pipelined steps (no L2 flush): frame record in with the launch, "
                       "count, then the points (lidar_points_download) out to pinned memory on a copy stream "
                       "two steps behind the casts, four device point buffers in rotation; consecutive casts "
                       "overlap (each starts on the SMs the previous one's last traversals leave idle); the "
                       "launch tuned for this regime (back-to-back casts, no flush)",
                "cast_overlap": L.cast_overlap(), "launch": stream_cfg},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "peak_source": f"{peaks_src} hbm_gbs (STREAM-style copy)",
                     "bytes_per_launch": visit_bytes, "kernel": "k_cast", "kernel_ms": kernel_ms,
                     "achieved_is": "the traversal's consumption rate of algorithmic bytes (node fetches x node "
                                    "size + triangle tests x 48 B + 17 B/ray I/O) against the HBM copy peak, the "
                                    "roofline model of the traversal; L1 and L2 serve most of these bytes, so this "
                                    "is not an HBM traffic rate (that is compulsory_frac and ncu_bytes_per_ray.dram)",
                     "binding_unit": (dict(NCU_UNITS, what="latency of dependent node fetches (L1/L2) and "
                                                           "instruction issue; fractions of one ncu-captured "
                                                           "launch of this kernel")
                                      if same_kernel else None),
                     "compulsory_bytes_per_launch": uniq_bytes,
                     # per ray from the same ncu capture: DRAM, L2 and L1 (global-load sector) bytes
                     "ncu_bytes_per_ray": ({"dram": traffic / n_beams,
                                            "l2": NCU_TRAFFIC["l2_bytes"] / n_beams,
                                            "l1_global_load": NCU_TRAFFIC["l1_global_load_bytes"] / n_beams}
                                           if same_kernel else None),
                     "compulsory_frac": uniq_bytes / (kernel_ms / 1e3) / 1e9 / hbm},
        "work_per_ray": {k: (v if k == "node_bytes" else v / n_beams) for k, v in counters.items()},
        "alu": {"bound": "alu", "flops_per_launch_ncu": NCU_FP32["fp32_flops"] if ncu_ok else None,
                "achieved_tflops_ncu": ncu_fp32_tf, "peak_tflops": fp_peak,
                "frac": (ncu_fp32_tf if ncu_ok else alu_tf) / fp_peak,
                "achieved_tops_alg": alu_tf,
                "peak_source": "measured: FP32 FMA probe kernel on this GPU, "
                               f"{fp_probe['tflops']:.1f} TFLOP/s at {fp_probe.get('sm_mhz')} MHz median, scaled "
                               f"to the {sm_mhz:.0f} MHz median of the timed casts",
                "probe": fp_probe,
                # the same measured rate at the maximum SM clock and at the median clock under a
                # long GEMM load recorded with the HBM and tensor peaks
                "peak_tflops_at_mhz": ({f"{mhz:.0f}": fp_probe["tflops"] * mhz / fp_probe["sm_mhz"]
                                        for mhz in (2070.0, float(peaks.get("clocks_under_load", {})
                                                                  .get("sm_mhz_median", 1455.0)))}
                                       if fp_probe.get("sm_mhz") else None),
                "ops_per_launch_alg": flops, "ops_per_launch_ncu": NCU_FP32["fp32_ops"] if ncu_ok else None,
                "ops": "alg: 20 FP32 ops per child box of a fetched node, 40 per triangle test (from the "
                       "source, each operation once); ncu: FP32 thread instructions of one captured launch "
                       "(sm__sass_thread_inst_executed_op_*_pred_on), each lane operation once (ops) or with "
                       "FMAs and packed pairs counted as two (flops, the unit of the measured peak)"},
        "clocks": clocks,
    }
    line.update(extras)
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"], ref = cpu_baseline(w, args, want_result=True)
        line["parity"] = parity_check(parity_dense, ref, w)
    if world > 1:
        torch.distributed.destroy_process_group()
    return line


TAPE_BYTES_PER_BEAM = 16  # valid 1 + mat 2 + theta 4 + rf 4 (tape) + intensity 4 + valid 1 (targets)


def cfg3_adjoint(torch, L, scene, use_cache=True):
    """cfg3 (16 frames of the 128-ch sensor): targets from the hidden table, the
    tape of a forward at the model's table, and closures for the forward, the
    fused-MSE backward alone and both.  The 16-frame cast is tuned on its own
    (a throughput workload: its best launch differs from a single frame's)."""
    import synth
    from paper_2208_10295_gb300.tune import autotune
    w3 = synth.cfg3()
    L.set_sensor(0, w3.sensors[0])
    L.set_materials(L.build_tables(torch.tensor(w3.params, device=L.device)))
    cfg3, _ = autotune(L, scene, w3.frames, w3.seed, schedule_frames=w3.frames[:1], use_cache=use_cache,
                       points=False)
    th = L.build_tables(torch.tensor(w3.hidden_params, device=L.device))
    tp = torch.tensor(w3.params, device=L.device)
    n3 = L.total_beams(w3.frames)
    tgt = L.alloc_beams(n3, ("valid", "intensity", "mat", "theta_deg", "rf"))
    L.set_materials(th)
    L.cast_into(scene, w3.frames, w3.seed, tgt)
    tape = L.alloc_beams(n3, ("valid", "intensity", "mat", "theta_deg", "rf"))
    loss = torch.zeros(1, device=L.device)
    gT = torch.zeros((tp.shape[0], 91), device=L.device)
    gg = torch.zeros(1, device=L.device)

    def fwd():
        T = L.build_tables(tp)
        L.set_materials(T)
        L.cast_into(scene, w3.frames, w3.seed, tape)
        return T

    def bwd():
        gT.zero_()
        gg.zero_()
        L.cast_backward_mse(tape, 1.0, tgt["intensity"], tgt["valid"], loss, gT, gg)
        L.build_tables_backward(tp, gT)

    def fwd_bwd():
        fwd()
        bwd()

    def bwd_kernel():
        L.cast_backward_mse(tape, 1.0, tgt["intensity"], tgt["valid"], loss, gT, gg)

    return {"n": n3, "fwd": fwd, "bwd": bwd, "fwd_bwd": fwd_bwd, "bwd_kernel": bwd_kernel, "loss": loss,
            "tape": tape, "targets": tgt, "launch": cfg3}


def run_extras(args, torch, L, scene, w1, table, flush, stream, single_step, tuned_cfg):
    import synth
    from paper_2208_10295_gb300.tune import apply as apply_cfg
    from paper_2208_10295_gb300.tune import autotune
    out = {}
    single_ms = event_time(torch, stream, single_step, flush, reps=20, warm=3)
    # ---- cfg2: 8 sensors x 64 frames as one CUDA graph replay
    w2 = synth.cfg2()
    for s, spec in enumerate(w2.sensors):
        L.set_sensor(s, spec)
    L.set_materials(table)
    first = np.concatenate([w2.frames[w2.frames["sensor"] == s][:1] for s in range(len(w2.sensors))])
    cfg2, _ = autotune(L, scene, w2.frames[: 8 * 4], w2.seed, schedule_frames=first, use_cache=not args.retune,
                       points=True)
    B = L.batch(w2.frames)
    pts2 = L.alloc_points(B.n_beams)
    poses = torch.tensor(np.stack([f["pose"] for f in w2.frames]), device=L.device)
    G = B.graph(scene, w2.seed, points=pts2, poses=poses)
    g_ms = event_time(torch, stream, G.launch, flush, reps=5, warm=2)
    out["batched"] = {"workload": "cfg2: 8 sensors (2x16, 2x32, 2x64, 1x128 spinning, 256x128 raster) x 64 frames, "
                                  "one CUDA-graph replay incl. pose upload and ordered compaction",
                      "rays_per_launch": B.n_beams, "ms_per_launch": g_ms,
                      "rays_per_s": B.n_beams / (g_ms / 1e3), "points": int(pts2["count"].item()),
                      "launch": cfg2}
    G.free()
    B.free()
    del pts2
    # ---- the paper's own raster-and-resample sampling on the same cfg1 frame, against the ray cast
    L.set_sensor(0, w1.sensors[0])
    near1 = w1.frames.copy()
    near1[0]["pose"][3] += 1.0
    near1[0]["pose"][7] += 0.5
    apply_cfg(L, scene, tuned_cfg, near1, w1.seed)
    fr1 = w1.frames
    nb1 = L.total_beams(fr1)
    rf = ("valid", "tri", "t")
    ref = L.alloc_beams(nb1, rf)
    L.cast_into(scene, fr1, w1.seed, ref)
    ref_np = {k: v.cpu().numpy() for k, v in ref.items()}
    cast_ms = event_time(torch, stream, lambda: L.cast_into(scene, fr1, w1.seed, ref), flush, reps=10, warm=3)
    ras = L.alloc_beams(nb1, rf)
    rows = []
    for width in (512, 1024, 2048):
        r_ms = event_time(torch, stream, lambda: L.raster_cast_into(scene, fr1, w1.seed, ras, width=width,
                                                                    n_cameras=6), flush, reps=10, warm=3)
        got = {k: v.cpu().numpy() for k, v in ras.items()}
        both = (got["tri"].view(np.uint32) != 0xFFFFFFFF) & (ref_np["tri"].view(np.uint32) != 0xFFFFFFFF)
        dt = np.abs(got["t"][both].astype(np.float64) - ref_np["t"][both])
        rows.append({"width": width, "n_cameras": 6, "ms_per_frame": r_ms, "rays_per_s": nb1 / (r_ms / 1e3),
                     "pixels_per_s": 6 * width * width / (r_ms / 1e3),
                     "same_triangle_frac": float((got["tri"][both] == ref_np["tri"][both]).mean()),
                     "range_err_m": {"median": float(np.median(dt)), "p90": float(np.percentile(dt, 90)),
                                     "p99": float(np.percentile(dt, 99)), "max": float(dt.max())},
                     "valid_agree_frac": float((got["valid"] == ref_np["valid"]).mean())})
    out["raster"] = {"workload": "cfg1 frame through the raster-and-resample path (6 pin-hole cameras, 24-bit "
                                 "depth/angle G-buffer), compared beam by beam with the ray cast of the same frame",
                     "ray_cast_ms_per_frame": cast_ms, "by_width": rows}
    del ref, ras
    # ---- rolling-shutter sweeps along the cfg3 trajectory vs the frame cast of the same poses
    w3s = synth.cfg3()
    L.set_sensor(0, w3s.sensors[0])
    sw = synth.make_sweep_frames([(0, int(a["frame"]), a["pose"], b["pose"])
                                  for a, b in zip(w3s.frames[:-1], w3s.frames[1:])])
    nsw = L.total_beams(sw)
    sbuf = L.alloc_beams(nsw, ("valid", "range", "intensity"))
    sw_ms = event_time(torch, stream, lambda: L.cast_sweep_into(scene, sw, w3s.seed, sbuf), flush, reps=5, warm=2)
    fr_ms = event_time(torch, stream, lambda: L.cast_into(scene, w3s.frames[:-1], w3s.seed, sbuf), flush, reps=5,
                       warm=2)
    out["rolling_shutter"] = {"workload": "15 sweeps of the 128-ch sensor along the 16-frame trajectory over the "
                                          "1.04M-tri scene, each beam at its own interpolated pose",
                              "beams": nsw, "sweep_ms": sw_ms, "rays_per_s": nsw / (sw_ms / 1e3),
                              "frame_cast_same_poses_ms": fr_ms}
    del sbuf
    L.set_sensor(0, w1.sensors[0])
    # ---- cfg3: 16 frames forward (dense tape) + fused-MSE adjoint vs plain forward
    d3 = cfg3_adjoint(torch, L, scene, use_cache=not args.retune)
    f_ms = event_time(torch, stream, d3["fwd"], flush, reps=10, warm=2)
    fb_ms = event_time(torch, stream, d3["fwd_bwd"], flush, reps=10, warm=2)
    b_ms = event_time(torch, stream, d3["bwd"], flush, reps=20, warm=3)
    # the backward kernel alone (the fused-MSE call, without clearing the
    # gradient buffers or the table-builder backward): the roofline's duration
    bk_ms = event_time(torch, stream, d3["bwd_kernel"], flush, reps=20, warm=3)
    # algorithmic bytes: the tape and the targets, read once
    b_bytes = TAPE_BYTES_PER_BEAM * d3["n"]
    hbm = float(load_peaks()[0].get("hbm_gbs", HBM_FALLBACK_GBS))
    out["differentiation"] = {"workload": "cfg3: 128-ch x 2048 az x 16 frames (4,194,304 beams), forward with tape + "
                                          "fused MSE adjoint to the 32x91 table, widths and gain",
                              "fwd_ms": f_ms, "fwd_bwd_ms": fb_ms, "bwd_ms": fb_ms - f_ms,
                              "bwd_alone_ms": b_ms, "plain_single_frame_fwd_ms": single_ms,
                              "loss": float(d3["loss"].item()), "launch": d3["launch"],
                              "bwd_kernel_ms": bk_ms,
                              "bwd_roofline": {"bound": "hbm", "achieved": b_bytes / (bk_ms / 1e3) / 1e9,
                                               "peak": hbm, "unit": "GB/s",
                                               "frac": b_bytes / (bk_ms / 1e3) / 1e9 / hbm,
                                               "bytes_per_launch": b_bytes, "kernel": "k_adj_onepass",
                                               "kernel_ms": bk_ms,
                                               "traffic": ADJ_TRAFFIC["bytes"]
                                               if ADJ_TRAFFIC["sources"] == adjoint_digest() else None,
                                               "note": "tape + targets, 16 B/beam, each read once by the "
                                                       "algorithm; the fused-MSE backward call alone, L2 "
                                                       "flushed before each; traffic from the ncu capture"}}
    L.set_materials(table)
    L.set_sensor(0, w1.sensors[0])
    del d3
    # ---- cfg4: the ~10.7M-triangle city, 128-ch x 4096 az x 32 frames x 7 sub-rays
    if not args.no_city:
        w4 = synth.cfg4()
        scene4 = build_city(L, w4)
        L.set_sensor(0, w4.sensors[0])
        t4 = L.build_tables(torch.tensor(w4.params, device=L.device))
        L.set_materials(t4)
        cfg4, _ = autotune(L, scene4, w4.frames[:4], w4.seed, schedule_frames=w4.frames[:1],
                           use_cache=not args.retune, points=True)
        B4 = L.batch(w4.frames)
        pts4 = L.alloc_points(B4.n_beams)
        c_ms = event_time(torch, stream, lambda: B4.cast_into(scene4, w4.seed, None, pts4), None, reps=3, warm=1)
        info = scene4.info()
        # traversal work of four frames (instrumented kernel), scaled to the 32-frame launch
        cw = L.count_work(scene4, w4.frames[:4], w4.seed)
        sub_bytes = (cw["node_visits"] * cw["node_bytes"] + cw["tri_tests"] * 48) / cw["rays"]
        city_bytes = sub_bytes * B4.n_beams * 7
        hbm = float(load_peaks()[0].get("hbm_gbs", HBM_FALLBACK_GBS))
        out["city"] = {"workload": "cfg4: 10.7M-tri city (4096 m terrain + 20,000 buildings), 128-ch x 4096 az x "
                                   "32 frames x 7 sub-rays (0.1 mrad), strongest return, ordered compaction",
                       "tris": int(w4.scene.n_tris), "beams": B4.n_beams, "subrays": B4.n_beams * 7,
                       "ms": c_ms, "subrays_per_s": B4.n_beams * 7 / (c_ms / 1e3),
                       "build_ms": info["build_ms"], "bvh_depth": info["max_depth"],
                       "tree": f"{tree_name(CITY_TREE)} ({info['treelets']} treelets rewritten)",
                       "points": int(pts4["count"].item()), "launch": cfg4,
                       "work_per_subray": {"node_visits": cw["node_visits"] / cw["rays"],
                                           "tri_tests": cw["tri_tests"] / cw["rays"],
                                           "node_bytes": cw["node_bytes"],
                                           "unique_bytes_4_frames": cw["unique_node_bytes"] + cw["unique_tri_bytes"]},
                       "traversal_bytes": {
                           "rate_gbs": city_bytes / (c_ms / 1e3) / 1e9, "bytes_per_launch": city_bytes,
                           "hbm_peak_gbs": hbm, "frac_of_hbm": None,
                           "note": "algorithmic node and triangle bytes of the traversal per sub-ray (from four "
                                   "frames), at a rate above the HBM copy peak: a beam's seven sub-rays and its "
                                   "neighbours walk the same nodes, so L1 serves ~93 % of them and no fraction of "
                                   "HBM is claimed; what binds is instruction issue",
                           "binding_unit": (dict(NCU_CITY_UNITS, source="ncu --set full of one city frame "
                                                                         "launch (profiles/k_cast_city_ncu_full.md)")
                                            if NCU_CITY_UNITS["sources"] == kernel_digest() and
                                            NCU_CITY_UNITS["tree"] == CITY_TREE and
                                            kernel_name(cfg4) == NCU_CITY_UNITS["kernel"] else None)}}
        # forward with tape (each beam's strongest sub-ray) + fused-MSE adjoint to the 64 x 91 table, the
        # widths and the gain, targets from the hidden table
        del pts4
        tf = ("valid", "intensity", "mat", "theta_deg", "rf")
        tgt4 = L.alloc_beams(B4.n_beams, tf)
        L.set_materials(L.build_tables(torch.tensor(w4.hidden_params, device=L.device)))
        B4.cast_into(scene4, w4.seed, tgt4)
        tape4 = L.alloc_beams(B4.n_beams, tf)
        tp4 = torch.tensor(w4.params, device=L.device)
        loss4 = torch.zeros(1, device=L.device)
        gT4 = torch.zeros((tp4.shape[0], 91), device=L.device)
        gg4 = torch.zeros(1, device=L.device)

        def fwd4():
            L.set_materials(L.build_tables(tp4))
            B4.cast_into(scene4, w4.seed, tape4)

        def fwd_bwd4():
            fwd4()
            gT4.zero_()
            gg4.zero_()
            L.cast_backward_mse(tape4, 1.0, tgt4["intensity"], tgt4["valid"], loss4, gT4, gg4)
            L.build_tables_backward(tp4, gT4)

        f4_ms = event_time(torch, stream, fwd4, None, reps=3, warm=1)
        fb4_ms = event_time(torch, stream, fwd_bwd4, None, reps=3, warm=1)
        out["city"]["forward_adjoint"] = {"workload": "cfg4: the 32 frames with tape (strongest sub-ray per beam) "
                                                      "+ fused-MSE adjoint to the 64x91 table, widths and gain",
                                          "fwd_ms": f4_ms, "fwd_bwd_ms": fb4_ms, "bwd_ms": fb4_ms - f4_ms,
                                          "loss": float(loss4.item())}
        del tgt4, tape4
        L.set_materials(t4)
        B4.free()
        # multi-echo (first and last of the 7 sub-ray returns, 0.5 m apart) over sweeps of the same trajectory
        sw4 = synth.make_sweep_frames([(0, int(a["frame"]), a["pose"], b["pose"])
                                       for a, b in zip(w4.frames[:-1], w4.frames[1:])])
        n4 = L.total_beams(sw4)
        e4 = L.alloc_echoes(n4, 2)
        e_ms = event_time(torch, stream, lambda: L.cast_sweep_into(scene4, sw4, w4.seed, None, e4, mode=1,
                                                                   separation=0.5), None, reps=3, warm=1)
        cnt = e4["count"].cpu().numpy()
        out["city"]["echoes"] = {"workload": "31 sweeps x 524,288 beams x 7 sub-rays, first and last return "
                                             ">= 0.5 m apart", "ms": e_ms, "subrays_per_s": n4 * 7 / (e_ms / 1e3),
                                 "beams_with_return": int((cnt > 0).sum()), "beams_with_two": int((cnt > 1).sum())}
        del e4
        scene4.free()
        L.set_materials(table)
        L.set_sensor(0, w1.sensors[0])
    return out


def cpu_baseline(w, args, n_beams=None, want_result=False):
    import oracle
    oracle.build()
    nb = n_beams or args.cpu_beams
    sensor = w.sensors[0]
    rng = np.random.default_rng(123)
    beams = np.sort(rng.choice(sensor.n_beams, nb, replace=False)).astype(np.int64)
    samples = (np.zeros(nb, np.int64), beams)
    T = oracle.build_tables(w.params)
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    ref = oracle.cast(w.scene, w.sensors, w.frames, T, w.seed, samples=samples, n_threads=cores)
    dt = time.perf_counter() - t0
    cb = {"value": nb / dt, "unit": UNIT, "cores": cores, "per_core": nb / dt / cores, "kind": "oracle",
          "sample": f"{nb} seeded beams of the same frame (brute force FP64 over all {w.scene.n_tris} tris), "
                    f"{dt:.1f} s"}
    return (cb, ref) if want_result else cb


def parity_check(dense, ref, w):
    """The timed frame's dense GPU records against the oracle on the CPU
    baseline's sample of beams (untimed): exemption counts and largest errors,
    with the tolerances of the parity tests."""
    if dense is None:
        return None
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import compare
    idx = ref["sample_beam"]
    got = {k: (v.view(np.uint32) if k in ("tri", "inst") else (v.view(np.uint16) if k == "mat" else v))[idx]
           for k, v in dense.items()}
    try:
        rep = compare(got, ref, gain=max(s.gain for s in w.sensors), label="cfg1 frame, CPU-baseline sample")
        rep["ok"] = True
    except AssertionError as e:
        rep = {"ok": False, "mismatch": str(e), "beams": int(idx.size)}
    rep["tolerances"] = "tri, instance, material, valid bit-exact outside counted exemptions; range rel 1e-5; " \
                        "intensity rel 1e-4 (floor 1e-7 g); normal abs 1e-5"
    return rep


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import synth
    w = synth.cfg1()
    for _ in range(args.warmup):
        cpu_baseline(w, args, n_beams=64)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, args, n_beams=args.ref_beams))
    total = time.perf_counter() - t0
    value = args.ref_beams * args.steps / total
    cb = vals[-1]
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "cfg1: 128-ch x 2048 az over the 1,036,288-tri scene; each step a bounded "
                                   f"sample of {args.ref_beams} beams"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"], "per_core": value / cb["cores"],
                             "kind": "oracle", "sample": f"{args.ref_beams} seeded beams per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-beams", type=int, default=16384,
                    help="beams of the oracle's timed sample (about 13 s on 16 cores)")
    ap.add_argument("--ref-beams", type=int, default=None,
                    help="beams per reference-arm step (default: about 90 s of oracle work over all steps)")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg (profiling runs)")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched/differentiation/city measurements")
    ap.add_argument("--no-city", action="store_true", help="skip the 10.7M-triangle city measurement")
    ap.add_argument("--raster-only", action="store_true",
                    help="time only the raster-and-resample path on the cfg1 frame (warmup + steps calls) and exit")
    ap.add_argument("--city-only", action="store_true",
                    help="time only the cast of one city frame with 7 sub-rays (warmup + steps launches) and exit")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the cfg3 fused-MSE backward (warmup + steps calls) and exit")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time only the cast kernel of the roofline (warmup + steps launches) and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.ref_beams is None:
        # the oracle does ~1,250 beams/s of this frame on 16 cores: bound the whole reference run
        args.ref_beams = int(min(4096, max(16, 90 * 1250 // max(args.steps, 1))))
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local_rank)
    if rank == 0 and line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
