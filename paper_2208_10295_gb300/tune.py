"""Autotuner for the cast kernel's launch configuration and ray schedule.

Searches threads per block x resident blocks per SM (which also picks the
register budget: up to 512 threads per SM 128 registers, up to 768 85, more
64), the traversal variant, the ray order (beam order / Morton
order of directions), the schedule (Morton groups / most expensive groups
first / per-beam cost buckets) and, when the point cloud is timed too, whether
the ordered scatter runs inside the cast (cooperative launch) or as its own
kernel, timing each candidate with CUDA events on the context stream.  Every
candidate produces bit-identical results (tested), so the choice is purely a
performance one.  The winner is cached in a JSON file keyed by GPU name, SM
count and a hash of the workload's shape and of its hierarchy's size.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
import statistics

import numpy as np
import torch

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")

SPACE = {
    "block_threads": (64, 128, 256),
    "blocks_per_sm": (2, 3, 4, 6, 8, 12),
    "traversal": (0, 1, 2, 3),
    "ray_order": (0, 1),
    "schedule": ("morton", "cost", "bucket"),
    "fused_scatter": (0, 1),
}


def workload_key(L, scene, frames) -> str:
    props = torch.cuda.get_device_properties(L.device)
    fr = np.ascontiguousarray(frames)
    info = scene.info()
    # the hierarchy as well as the sizes: a tree built with other options
    # (another method, treelet rounds) is another workload
    shape = ([int(scene.n_tris), int(info["n_nodes4"]), int(info["n_nodes8"]), int(info["treelets"])] +
             [int(L.n_beams[int(s)]) for s in fr["sensor"]])
    h = hashlib.sha256(json.dumps(shape).encode()).hexdigest()[:16]
    return f"{props.name}|{props.multi_processor_count}|{h}"


def _time_cast(L, scene, frames, seed, out, pts, flush, reps):
    ts = []
    stream = L.stream
    for i in range(reps + 2):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        L.cast_into(scene, frames, seed, out, pts)
        b.record(stream)
        b.synchronize()
        if i >= 2:
            ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def _time_stream(L, scene, frames, seed, pts_list, reps):
    """Per-cast time of back-to-back casts into rotating point buffers (no L2
    flush; consecutive casts overlap): the streaming regime."""
    stream = L.stream
    ts = []
    for i in range(reps + 1):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(8):
            L.cast_into(scene, frames, seed, None, pts_list[k % len(pts_list)])
        b.record(stream)
        b.synchronize()
        if i >= 1:
            ts.append(a.elapsed_time(b) / 8)
    return statistics.median(ts)


def candidates(points=False, wide8=True, restrict=None):
    """Every valid configuration of SPACE; `restrict` (key -> allowed values)
    narrows the search to part of it."""
    space = {k: tuple(v for v in vals if restrict is None or k not in restrict or v in restrict[k])
             for k, vals in SPACE.items()}
    for bt, bps, tv, ro, sc, fs in itertools.product(*space.values()):
        if bt * bps > 2048 or bt * bps < 256:
            continue
        if tv == 3 and not wide8:
            continue  # the scene kept no 8-wide tree
        if ro == 0 and sc != "morton":
            continue  # the cost schedules reorder the Morton order
        if not points and fs == 0:
            continue  # without a point cloud there is no scatter
        yield {"block_threads": bt, "blocks_per_sm": bps, "tile_rays": 32, "traversal": tv, "ray_order": ro,
               "fused_scatter": fs, "schedule": sc}


def apply(L, scene, cfg, schedule_frames, seed):
    L.set_launch_config(**{k: v for k, v in cfg.items() if k != "schedule"})
    slots = sorted({int(s) for s in np.ascontiguousarray(schedule_frames)["sensor"]})
    for s in slots:
        L.reset_schedule(s)
    if cfg.get("schedule") in ("cost", "bucket"):
        fr = np.ascontiguousarray(schedule_frames)
        for s in slots:
            first = fr[fr["sensor"] == s][:1]
            L.schedule_by_cost(scene, first, seed, mode=0 if cfg["schedule"] == "cost" else 1)


def autotune(L, scene, frames, seed, schedule_frames=None, cache_path=DEFAULT_CACHE, reps=8, flush_l2=True,
             use_cache=True, verbose=False, points=False, restrict=None, streaming=False):
    """Picks and applies the fastest configuration for casting `frames`
    (`points`: the cast plus the ordered compaction into a point cloud,
    otherwise the cast to dense valid flags).  `schedule_frames` (default
    `frames`) are the poses whose measured costs order the rays for the cost
    schedules: pass a nearby pose (the previous frame) to keep the
    measurement honest.  `restrict` (key -> allowed values) narrows the
    search.  `streaming`: time back-to-back casts of the frames into rotating
    point buffers without an L2 flush (a sensor streaming frames; consecutive
    casts overlap) instead of one flushed cast.  Returns (config, ms)."""
    schedule_frames = frames if schedule_frames is None else schedule_frames
    key = workload_key(L, scene, frames) + ("|points" if points else "|dense")
    if restrict:
        key += "|" + json.dumps({k: list(v) for k, v in sorted(restrict.items())})
    if streaming:
        key += "|stream"
    cache = {}
    if use_cache and cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    if use_cache and key in cache:
        cfg = cache[key]["config"]
        apply(L, scene, cfg, schedule_frames, seed)
        return cfg, cache[key]["ms"]
    n = L.total_beams(frames)
    out = None if points else L.alloc_beams(n, ("valid",))
    pts = L.alloc_points(n) if points else None
    pts_list = [pts] + [L.alloc_points(n) for _ in range(2)] if streaming else None
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=L.device) if flush_l2 else None
    best = None
    for cfg in candidates(points, wide8=scene.info()["n_nodes8"] > 0 or scene.n_tris == 0, restrict=restrict):
        apply(L, scene, cfg, schedule_frames, seed)
        ms = (_time_stream(L, scene, frames, seed, pts_list, max(reps // 2, 3)) if streaming
              else _time_cast(L, scene, frames, seed, out, pts, flush, reps))
        if verbose:
            print(f"{ms * 1e3:9.1f} us  {cfg}", flush=True)
        if best is None or ms < best[1]:
            best = (cfg, ms)
    apply(L, scene, best[0], schedule_frames, seed)
    if cache_path:
        cache[key] = {"config": best[0], "ms": best[1]}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best
