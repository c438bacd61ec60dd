"""PyTorch-facing wrapper over the C ABI: tensors in, tensors out.

Only argument marshalling happens here (device pointers, struct packing,
the current CUDA stream); every step of the per-beam model runs in the CUDA
library.  `LidarCast` is a torch.autograd.Function whose backward calls the
library's adjoint kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi as C

FRAME_DTYPE = np.dtype([("sensor", np.int32), ("frame", np.int32), ("pose", np.float32, (12,))])


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _frames_array(frames):
    fr = np.ascontiguousarray(frames)
    if fr.dtype != FRAME_DTYPE:
        fr = fr.astype(FRAME_DTYPE)
    return fr


class Scene:
    def __init__(self, lidar, handle, n_tris):
        self._lidar = lidar
        self.handle = handle
        self.n_tris = n_tris

    def info(self):
        info = C.lidar_scene_info()
        C.check(C.lidar_get_scene_info(self.handle, ctypes.byref(info)), "lidar_get_scene_info")
        return {k: getattr(info, k) for k, _ in info._fields_}

    def export(self):
        info = self.info()
        nodes = np.zeros((max(info["n_nodes"], 1), 16), np.float32)
        leaf = np.zeros(max(self.n_tris, 1), np.uint32)
        C.check(C.lidar_scene_export(self.handle, nodes.ctypes.data_as(ctypes.c_void_p),
                                     leaf.ctypes.data_as(ctypes.c_void_p)), "lidar_scene_export")
        return nodes[:info["n_nodes"]], leaf[:self.n_tris]

    def export_wide(self, width):
        """The 4- or 8-wide tree as float32 [n][8 * width] (device layout)."""
        n = self.info()["n_nodes4" if width == 4 else "n_nodes8"]
        nodes = np.zeros((max(n, 1), 8 * width), np.float32)
        C.check(C.lidar_scene_export_wide(self.handle, width, nodes.ctypes.data_as(ctypes.c_void_p)),
                "lidar_scene_export_wide")
        return nodes[:n]

    def free(self):
        if self.handle is not None and self._lidar.handle is not None:
            C.lidar_scene_free(self.handle)
        self.handle = None


class Lidar:
    """One library context bound to a CUDA device and stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream = None):
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        C.check(C.lidar_create(device, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "lidar_create")
        self.handle = h
        self.n_beams = {}
        self.gains = {}
        self._keep = []
        self._table = None

    def close(self):
        if self.handle is not None:
            C.lidar_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- scene
    def build_scene(self, verts, tris, mat=None, inst=None) -> Scene:
        verts = torch.as_tensor(verts, dtype=torch.float32, device=self.device).contiguous()
        tris = torch.as_tensor(np.asarray(tris).astype(np.int32) if isinstance(tris, np.ndarray) else tris,
                               device=self.device).to(torch.int32).contiguous()
        n = tris.shape[0]
        mat_t = None if mat is None else torch.as_tensor(np.asarray(mat).astype(np.int16), device=self.device)
        inst_t = None if inst is None else torch.as_tensor(np.asarray(inst).astype(np.int32), device=self.device)
        h = ctypes.c_void_p()
        C.check(C.lidar_scene_build(self.handle, _ptr(verts), verts.shape[0], _ptr(tris), n, _ptr(mat_t),
                                    _ptr(inst_t), ctypes.byref(h)), "lidar_scene_build")
        return Scene(self, h, n)

    # ----------------------------------------------------------- sensors
    def set_sensor(self, slot: int, spec):
        az = np.ascontiguousarray(spec.az_rad, dtype=np.float64)
        el = np.ascontiguousarray(spec.el_rad, dtype=np.float64)
        d = C.lidar_sensor_desc(az.size, az.ctypes.data, el.ctypes.data, spec.r_min, spec.r_max, spec.d_max,
                                spec.RL_max, spec.sigma, spec.gain, spec.range_exp, spec.r_ref,
                                spec.divergence_rad, spec.n_subrays, getattr(spec, "sigma_k", 0.0))
        C.check(C.lidar_set_sensor(self.handle, slot, ctypes.byref(d)), "lidar_set_sensor")
        self.n_beams[slot] = az.size
        self.gains[slot] = float(np.float32(spec.gain))

    def set_sensor_gain(self, slot: int, gain: float):
        C.check(C.lidar_set_sensor_gain(self.handle, slot, float(gain)), "lidar_set_sensor_gain")
        self.gains[slot] = float(np.float32(gain))

    def beam_dirs(self, slot: int) -> np.ndarray:
        out = np.zeros((self.n_beams[slot], 3), np.float32)
        C.check(C.lidar_get_beam_dirs(self.handle, slot, out.ctypes.data_as(ctypes.c_void_p)), "lidar_get_beam_dirs")
        return out

    # ----------------------------------------------------------- materials
    def build_tables(self, params: torch.Tensor) -> torch.Tensor:
        params = params.to(self.device, torch.float32).contiguous()
        M = params.shape[0]
        table = torch.empty((M, C.LIDAR_TABLE_SIZE), dtype=torch.float32, device=self.device)
        C.check(C.lidar_build_tables(self.handle, _ptr(params), M, _ptr(table)), "lidar_build_tables")
        return table

    def build_tables_backward(self, params: torch.Tensor, grad_table: torch.Tensor) -> torch.Tensor:
        params = params.to(self.device, torch.float32).contiguous()
        grad_table = grad_table.to(self.device, torch.float32).contiguous()
        out = torch.empty_like(params)
        C.check(C.lidar_build_tables_backward(self.handle, _ptr(params), _ptr(grad_table), params.shape[0],
                                              _ptr(out)), "lidar_build_tables_backward")
        return out

    def set_materials(self, table: torch.Tensor):
        table = table.to(self.device, torch.float32).contiguous()
        C.check(C.lidar_set_materials(self.handle, _ptr(table), table.shape[0]), "lidar_set_materials")
        self._table = table  # the library reads it in place: keep it alive

    # ----------------------------------------------------------- cast
    def total_beams(self, frames) -> int:
        """Beams of all frames (frame records or sweep records)."""
        fr = np.atleast_1d(np.asarray(frames))
        return int(sum(self.n_beams[int(s)] for s in fr["sensor"]))

    def alloc_beams(self, n: int, fields=("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst",
                                          "sub", "theta_deg", "rf")):
        dt = {"valid": torch.uint8, "tri": torch.int32, "t": torch.float32, "range": torch.float32,
              "intensity": torch.float32, "normal": torch.float32, "mat": torch.int16, "inst": torch.int32,
              "sub": torch.uint8, "theta_deg": torch.float32, "rf": torch.float32}
        out = {}
        for f in fields:
            shape = (n, 3) if f == "normal" else (n,)
            out[f] = torch.empty(shape, dtype=dt[f], device=self.device)
        return out

    def alloc_points(self, capacity: int):
        return {"xyz": torch.empty((capacity, 3), dtype=torch.float32, device=self.device),
                "range": torch.empty(capacity, dtype=torch.float32, device=self.device),
                "intensity": torch.empty(capacity, dtype=torch.float32, device=self.device),
                "normal": torch.empty((capacity, 3), dtype=torch.float32, device=self.device),
                "material": torch.empty(capacity, dtype=torch.int16, device=self.device),
                "instance": torch.empty(capacity, dtype=torch.int32, device=self.device),
                "beam": torch.empty(capacity, dtype=torch.int32, device=self.device),
                "frame": torch.empty(capacity, dtype=torch.int32, device=self.device),
                "count": torch.zeros(1, dtype=torch.int64, device=self.device)}

    @staticmethod
    def beams_struct(b):
        s = C.lidar_beams()
        for name, _ in s._fields_:
            t = b.get(name) if b is not None else None
            setattr(s, name, None if t is None else t.data_ptr())
        return s

    @staticmethod
    def points_struct(p):
        s = C.lidar_points()
        s.capacity = p["xyz"].shape[0] if p.get("xyz") is not None else p["range"].shape[0]
        for name, _ in s._fields_[1:]:
            t = p.get(name)
            setattr(s, name, None if t is None else t.data_ptr())
        return s

    def cast_into(self, scene: Scene, frames, seed: int, beams=None, points=None):
        fr = _frames_array(frames)
        bs = self.beams_struct(beams) if beams is not None else None
        ps = self.points_struct(points) if points is not None else None
        st = C.lidar_cast(self.handle, scene.handle, fr.ctypes.data_as(ctypes.c_void_p), len(fr),
                          ctypes.c_uint64(seed), ctypes.byref(bs) if bs is not None else None,
                          ctypes.byref(ps) if ps is not None else None,
                          _ptr(points["count"]) if points is not None else None)
        C.check(st, "lidar_cast")

    def download_points(self, points, host, count: int, stream=None):
        """Queues the copy of the first `count` points of every field present in
        both `points` (device tensors of a cast) and `host` (host tensors,
        pinned for asynchronous copies) on `stream` (default: the context's
        stream); one native call for all fields."""
        ds, hs = self.points_struct(points), self.points_struct(host)
        sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        C.check(C.lidar_points_download(self.handle, ctypes.byref(ds), ctypes.byref(hs), int(count), sp),
                "lidar_points_download")

    def cast(self, scene: Scene, frames, seed: int, dense=True, points_capacity=None):
        """Returns (beams dict, points dict or None)."""
        n = self.total_beams(frames)
        beams = self.alloc_beams(n) if dense else None
        points = self.alloc_points(points_capacity) if points_capacity is not None else None
        self.cast_into(scene, frames, seed, beams, points)
        return beams, points

    # ----------------------------------------------------------- batches / graphs
    def batch(self, frames) -> "Batch":
        fr = _frames_array(frames)
        h = ctypes.c_void_p()
        C.check(C.lidar_batch_create(self.handle, fr.ctypes.data_as(ctypes.c_void_p), len(fr), ctypes.byref(h)),
                "lidar_batch_create")
        return Batch(self, h, fr)

    def sync_status(self) -> int:
        return C.lidar_sync_status(self.handle)

    # ----------------------------------------------------------- adjoint
    def cast_backward(self, tape, gain: float, grad_I: torch.Tensor, grad_table: torch.Tensor,
                      grad_gain: torch.Tensor):
        n = tape["valid"].shape[0]
        ts = self.beams_struct(tape)
        C.check(C.lidar_cast_backward(self.handle, n, ctypes.byref(ts), float(gain), _ptr(grad_I.contiguous()),
                                      _ptr(grad_table), _ptr(grad_gain)), "lidar_cast_backward")

    def cast_backward_mse(self, tape, gain: float, target_I, target_valid, loss, grad_table, grad_gain,
                          n_used: torch.Tensor = None):
        """Fused-MSE adjoint; `n_used` (int64 [1] on the device, optional)
        receives the number of beams the mean runs over (for combining the
        partial results of ranks, `combine_mse` / `allreduce_mse`)."""
        n = tape["valid"].shape[0]
        ts = self.beams_struct(tape)
        if n_used is None:
            C.check(C.lidar_cast_backward_mse(self.handle, n, ctypes.byref(ts), float(gain), _ptr(target_I),
                                              _ptr(target_valid), _ptr(loss), _ptr(grad_table), _ptr(grad_gain)),
                    "lidar_cast_backward_mse")
        else:
            C.check(C.lidar_cast_backward_mse_count(self.handle, n, ctypes.byref(ts), float(gain), _ptr(target_I),
                                                    _ptr(target_valid), _ptr(loss), _ptr(grad_table),
                                                    _ptr(grad_gain), _ptr(n_used)),
                    "lidar_cast_backward_mse_count")

    def count_work(self, scene: Scene, frames, seed: int, beam_cost: torch.Tensor = None):
        """Work of one cast (instrumented kernel): node fetches, triangle tests,
        distinct nodes/triangles touched, and the bytes they stand for.
        `beam_cost` (int32 [n_beams], optional) receives each beam's cost."""
        fr = _frames_array(frames)
        wc = C.lidar_work_counts()
        C.check(C.lidar_count_work(self.handle, scene.handle, fr.ctypes.data_as(ctypes.c_void_p), len(fr),
                                   ctypes.c_uint64(seed), ctypes.byref(wc), _ptr(beam_cost)), "lidar_count_work")
        d = {k: int(getattr(wc, k)) for k, _ in wc._fields_}
        d["unique_node_bytes"] = d["unique_nodes"] * d["node_bytes"]
        d["unique_tri_bytes"] = d["unique_tris"] * 48
        # per ray: beam direction and ray-order index in, one valid byte out
        d["io_bytes"] = d["rays"] * (12 + 4 + 1)
        return d

    def schedule_by_cost(self, scene: Scene, frame, seed: int, mode: int = 0):
        """Most-expensive-first ray order from the costs measured on `frame`
        (one frame record of the slot to reschedule); mode 0 orders 32-beam
        groups, mode 1 single beams by cost bucket."""
        fr = _frames_array(frame).reshape(-1)[:1]
        C.check(C.lidar_schedule_by_cost(self.handle, scene.handle, fr.ctypes.data_as(ctypes.POINTER(C.lidar_frame)),
                                         ctypes.c_uint64(seed), int(mode)), "lidar_schedule_by_cost")

    def reset_schedule(self, slot: int):
        C.check(C.lidar_reset_schedule(self.handle, slot), "lidar_reset_schedule")

    # ----------------------------------------------------------- sweeps and echoes
    def alloc_echoes(self, n: int, n_echoes: int):
        return {"count": torch.empty(n, dtype=torch.uint8, device=self.device),
                "range": torch.empty((n, n_echoes), dtype=torch.float32, device=self.device),
                "intensity": torch.empty((n, n_echoes), dtype=torch.float32, device=self.device),
                "tri": torch.empty((n, n_echoes), dtype=torch.int32, device=self.device),
                "sub": torch.empty((n, n_echoes), dtype=torch.uint8, device=self.device)}

    def cast_sweep_into(self, scene: Scene, sweeps, seed: int, beams=None, echoes=None, mode: int = 0,
                        separation: float = 1.0):
        """Rolling-shutter cast of sweeps (records with sensor, frame, pose0,
        pose1), with optional multi-echo outputs (alloc_echoes)."""
        fr = np.ascontiguousarray(sweeps)
        assert fr.dtype.itemsize == 104
        bs = self.beams_struct(beams) if beams is not None else None
        es = None
        if echoes is not None:
            es = C.lidar_echoes(int(echoes["range"].shape[1]), mode, separation,
                                *[_ptr(echoes[k]) for k in ("count", "range", "intensity", "tri", "sub")])
        C.check(C.lidar_cast_sweep(self.handle, scene.handle, fr.ctypes.data_as(ctypes.c_void_p), len(fr),
                                   ctypes.c_uint64(seed), ctypes.byref(bs) if bs is not None else None,
                                   ctypes.byref(es) if es is not None else None), "lidar_cast_sweep")

    # ----------------------------------------------------------- raster path
    def raster_cast_into(self, scene: Scene, frames, seed: int, beams, width: int = 1024, n_cameras: int = 6):
        """The paper's raster-and-resample sampling (K pin-hole cameras of
        W x W pixels per frame, quantised G-buffer, each beam reading its pixel)
        into dense beam buffers."""
        fr = _frames_array(frames)
        cfg = C.lidar_raster_config(width, n_cameras)
        C.check(C.lidar_raster_cast(self.handle, scene.handle, fr.ctypes.data_as(ctypes.c_void_p), len(fr),
                                    ctypes.c_uint64(seed), ctypes.byref(cfg), ctypes.byref(self.beams_struct(beams))),
                "lidar_raster_cast")

    def raster_gbuffer(self, scene: Scene, frame, width: int = 1024, n_cameras: int = 6):
        """One frame's G-buffer: dict of [K, W, W] int32 tensors depth (24-bit
        code), angle_mat (24-bit angle code | stencil << 24), inst, tri."""
        fr = _frames_array(frame).reshape(-1)[:1]
        shape = (n_cameras, width, width)
        g = {k: torch.empty(shape, dtype=torch.int32, device=self.device)
             for k in ("depth", "angle_mat", "inst", "tri")}
        cfg = C.lidar_raster_config(width, n_cameras)
        C.check(C.lidar_raster_gbuffer(self.handle, scene.handle, fr.ctypes.data_as(ctypes.POINTER(C.lidar_frame)),
                                       ctypes.byref(cfg), *[_ptr(g[k]) for k in ("depth", "angle_mat", "inst", "tri")]),
                "lidar_raster_gbuffer")
        return g

    # ----------------------------------------------------------- build options
    def set_build_options(self, method: int = 1, ploc_radius: int = 16, collapse: int = None, tri_cost: float = None,
                          treelet_rounds: int = None, area_weight=None):
        """Hierarchy of scenes built afterwards: 0 Karras LBVH, 1 PLOC (default);
        `treelet_rounds` rounds of treelet restructuring of the binary tree;
        wide-node children by the largest-area rule (collapse 0) or the SAH
        dynamic program (collapse 1); `tri_cost` is a triangle test's cost
        relative to a node visit in both surface-area programs; `area_weight`
        (x, y, z) weights a box's faces in every area the builders compare.
        Options not given keep their current values."""
        cur = self.build_options()
        aw = cur["area_weight"] if area_weight is None else tuple(float(v) for v in area_weight)
        o = C.lidar_build_options(method, ploc_radius, cur["collapse"] if collapse is None else collapse,
                                  cur["tri_cost"] if tri_cost is None else tri_cost,
                                  cur["treelet_rounds"] if treelet_rounds is None else treelet_rounds,
                                  (ctypes.c_float * 3)(*aw))
        C.check(C.lidar_set_build_options(self.handle, ctypes.byref(o)), "lidar_set_build_options")

    def build_options(self):
        o = C.lidar_build_options()
        C.check(C.lidar_get_build_options(self.handle, ctypes.byref(o)), "lidar_get_build_options")
        return {"method": o.method, "ploc_radius": o.ploc_radius, "collapse": o.collapse, "tri_cost": o.tri_cost,
                "treelet_rounds": o.treelet_rounds, "area_weight": tuple(o.area_weight)}

    # ----------------------------------------------------------- tuning
    def launch_config(self):
        c = C.lidar_launch_config()
        C.check(C.lidar_get_launch_config(self.handle, ctypes.byref(c)), "lidar_get_launch_config")
        return {k: getattr(c, k) for k, _ in c._fields_}

    def set_launch_config(self, **kw):
        cur = self.launch_config()
        cur.update(kw)
        c = C.lidar_launch_config(**cur)
        C.check(C.lidar_set_launch_config(self.handle, ctypes.byref(c)), "lidar_set_launch_config")

    def wait_limit(self) -> int:
        """Limit (ns) of the bounded device-side waits."""
        v = ctypes.c_uint64()
        C.check(C.lidar_get_wait_limit(self.handle, ctypes.byref(v)), "lidar_get_wait_limit")
        return int(v.value)

    def measure_fp32_rate(self, fma_per_thread: int = 1 << 23) -> dict:
        """FP32 FMA rate of the device (FLOP/s, 2 per FMA) and the probe's kernel time."""
        r, t, pk = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        C.check(C.lidar_measure_fp32_rate(self.handle, int(fma_per_thread), ctypes.byref(r), ctypes.byref(t),
                                          ctypes.byref(pk)), "lidar_measure_fp32_rate")
        return {"flops_per_s": r.value, "kernel_ms": t.value, "packed": bool(pk.value)}

    def cast_overlap(self) -> bool:
        v = ctypes.c_int32()
        C.check(C.lidar_get_cast_overlap(self.handle, ctypes.byref(v)), "lidar_get_cast_overlap")
        return bool(v.value)

    def set_cast_overlap(self, enable: bool):
        """Consecutive direct casts may overlap (bit-identical results either way)."""
        C.check(C.lidar_set_cast_overlap(self.handle, int(bool(enable))), "lidar_set_cast_overlap")

    def set_wait_limit(self, ns: int):
        C.check(C.lidar_set_wait_limit(self.handle, int(ns)), "lidar_set_wait_limit")


class Batch:
    """Device-resident frames: casts without host copies, CUDA-graph capture."""

    def __init__(self, lidar, handle, frames):
        self._lidar = lidar
        self.handle = handle
        self.frames = frames
        self.n_beams = lidar.total_beams(frames)
        self._graphs = []

    def set_poses(self, poses: torch.Tensor):
        poses = poses.to(self._lidar.device, torch.float32).contiguous()
        C.check(C.lidar_batch_set_poses(self._lidar.handle, self.handle, _ptr(poses)), "lidar_batch_set_poses")

    def cast_into(self, scene: Scene, seed: int, beams=None, points=None):
        L = self._lidar
        bs = L.beams_struct(beams) if beams is not None else None
        ps = L.points_struct(points) if points is not None else None
        C.check(C.lidar_cast_batch(L.handle, scene.handle, self.handle, ctypes.c_uint64(seed),
                                   ctypes.byref(bs) if bs is not None else None,
                                   ctypes.byref(ps) if ps is not None else None,
                                   _ptr(points["count"]) if points is not None else None), "lidar_cast_batch")

    def graph(self, scene: Scene, seed: int, beams=None, points=None, poses: torch.Tensor = None) -> "Graph":
        L = self._lidar
        bs = L.beams_struct(beams) if beams is not None else None
        ps = L.points_struct(points) if points is not None else None
        h = ctypes.c_void_p()
        C.check(C.lidar_graph_create(L.handle, scene.handle, self.handle, _ptr(poses), ctypes.c_uint64(seed),
                                     ctypes.byref(bs) if bs is not None else None,
                                     ctypes.byref(ps) if ps is not None else None,
                                     _ptr(points["count"]) if points is not None else None, ctypes.byref(h)),
                "lidar_graph_create")
        g = Graph(L, h, keep=(beams, points, poses))
        self._graphs.append(g)
        return g

    def free(self):
        for g in self._graphs:
            g.free()
        if self.handle is not None and self._lidar.handle is not None:
            C.lidar_batch_free(self.handle)
        self.handle = None


class Graph:
    def __init__(self, lidar, handle, keep):
        self._lidar = lidar
        self.handle = handle
        self._keep = keep  # tensors baked into the graph stay alive with it

    def launch(self):
        C.check(C.lidar_graph_launch(self.handle), "lidar_graph_launch")

    def free(self):
        if self.handle is not None and self._lidar.handle is not None:
            C.lidar_graph_free(self.handle)
        self.handle = None


class LidarCast(torch.autograd.Function):
    """Intensities of every beam as a differentiable function of the material
    parameters (a, s, w) [M,3] and the sensor gain, with hits and masks held
    fixed from the forward pass (the per-beam model of Sec. II with the
    table builder in front of it).  The gain is that of one sensor slot, so
    every frame must name that slot (frames of other slots would keep their
    own gains in the forward pass while the backward applied this one)."""

    @staticmethod
    def forward(ctx, params, gain, lidar: Lidar, scene: Scene, frames, seed: int, slot: int):
        fr = _frames_array(frames)
        if np.any(fr["sensor"] != slot):
            raise ValueError(f"LidarCast differentiates the gain of sensor slot {slot}: every frame must name it")
        table = lidar.build_tables(params.detach())
        lidar.set_materials(table)
        lidar.set_sensor_gain(slot, float(gain.detach().cpu()))
        n = lidar.total_beams(frames)
        tape = lidar.alloc_beams(n, ("valid", "intensity", "mat", "theta_deg", "rf"))
        lidar.cast_into(scene, frames, seed, tape)
        ctx.lidar, ctx.tape, ctx.table, ctx.slot = lidar, tape, table, slot
        ctx.save_for_backward(params.detach(), gain.detach())
        I = tape["intensity"].clone()
        ctx.mark_non_differentiable(tape["valid"])
        return I, tape["valid"]

    @staticmethod
    def backward(ctx, grad_I, _grad_valid):
        params, gain = ctx.saved_tensors
        lidar = ctx.lidar
        lidar.set_materials(ctx.table)
        gT = torch.zeros_like(ctx.table)
        gg = torch.zeros(1, dtype=torch.float32, device=lidar.device)
        lidar.cast_backward(ctx.tape, float(gain), grad_I.contiguous().float(), gT, gg)
        gp = lidar.build_tables_backward(params, gT)
        return gp, gg.reshape(gain.shape), None, None, None, None, None


# ------------------------------------------------------- data-parallel fitting
#
# When the beams of one batch (frames of a trajectory) are split over ranks,
# each rank runs the fused-MSE adjoint over its own beams, into zeroed
# gradient buffers, with `n_used` counting the beams its mean ran over.  The
# batch's mean-squared loss and gradients are the partial results weighted by
# their counts: sum_r N_r x_r / sum_r N_r.  `combine_mse` does that for a list
# of partials held by one process; `allreduce_mse` does it across the ranks of
# a torch.distributed group with one all-reduce (FP64) of the weighted vector
# [N L, N dL/dT, N dL/dg, N] — the one exchange step of a sharded fit.

def _mse_vector(loss, grad_table, grad_gain, n_used):
    n = n_used.reshape(1).to(torch.float64)
    return torch.cat([loss.reshape(1).double() * n, grad_table.reshape(-1).double() * n,
                      grad_gain.reshape(1).double() * n, n])


def _mse_unpack(vec, loss, grad_table, grad_gain):
    N = vec[-1]
    scale = torch.where(N > 0, 1.0 / N, torch.zeros_like(N))
    loss.copy_((vec[0] * scale).reshape(loss.shape).to(loss.dtype))
    k = grad_table.numel()
    grad_table.copy_((vec[1:1 + k] * scale).reshape(grad_table.shape).to(grad_table.dtype))
    grad_gain.copy_((vec[1 + k] * scale).reshape(grad_gain.shape).to(grad_gain.dtype))
    return N


def combine_mse(parts, loss, grad_table, grad_gain):
    """Batch loss and gradients from per-part results `parts` = [(loss,
    grad_table, grad_gain, n_used), ...] (each over its own beams), written
    into loss, grad_table and grad_gain; returns the total count (a 0-d FP64
    tensor on the parts' device)."""
    vec = sum(_mse_vector(*p) for p in parts)
    return _mse_unpack(vec, loss, grad_table, grad_gain)


def allreduce_mse(loss, grad_table, grad_gain, n_used, group=None):
    """In place on every rank of `group`: this rank's loss, grad_table and
    grad_gain (over its own n_used beams) become the whole batch's; returns
    the batch's count (a 0-d FP64 tensor)."""
    import torch.distributed as dist
    vec = _mse_vector(loss, grad_table, grad_gain, n_used)
    dist.all_reduce(vec, op=dist.ReduceOp.SUM, group=group)
    return _mse_unpack(vec, loss, grad_table, grad_gain)
