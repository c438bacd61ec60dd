"""ctypes binding of include/lidar.h: the same names, argument marshalling only.

Every function here forwards to the compiled CUDA library; nothing computes on
the host.  A missing library raises immediately (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblidar.so")

LIDAR_OK = 0
LIDAR_EINVAL = -1
LIDAR_ENOMEM = -2
LIDAR_ECUDA = -3
LIDAR_ESTATE = -4
LIDAR_ESTACK = -5
LIDAR_ETIMEOUT = -6
LIDAR_ECAPACITY = -7
STATUS_NAMES = {0: "LIDAR_OK", -1: "LIDAR_EINVAL", -2: "LIDAR_ENOMEM", -3: "LIDAR_ECUDA", -4: "LIDAR_ESTATE",
                -5: "LIDAR_ESTACK", -6: "LIDAR_ETIMEOUT", -7: "LIDAR_ECAPACITY"}

LIDAR_NO_HIT = 0xFFFFFFFF
LIDAR_TABLE_SIZE = 91
LIDAR_MAX_SENSORS = 16
LIDAR_MAX_SUBRAYS = 8

c_vp = ctypes.c_void_p


class LidarError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lidar_scene_info(ctypes.Structure):
    _fields_ = [("n_tris", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("max_depth", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("build_ms", ctypes.c_double), ("n_nodes4", ctypes.c_int64),
                ("levels4", ctypes.c_int32), ("n_nodes8", ctypes.c_int64), ("levels8", ctypes.c_int32),
                ("treelets", ctypes.c_int64)]


class lidar_sensor_desc(ctypes.Structure):
    _fields_ = [("n_beams", ctypes.c_int64), ("az_rad", c_vp), ("el_rad", c_vp),
                ("r_min", ctypes.c_float), ("r_max", ctypes.c_float), ("d_max", ctypes.c_float),
                ("RL_max", ctypes.c_float), ("sigma", ctypes.c_float), ("gain", ctypes.c_float),
                ("range_exp", ctypes.c_float), ("r_ref", ctypes.c_float), ("divergence_rad", ctypes.c_float),
                ("n_subrays", ctypes.c_int32), ("sigma_k", ctypes.c_float)]


class lidar_frame(ctypes.Structure):
    _fields_ = [("sensor", ctypes.c_int32), ("frame", ctypes.c_int32), ("pose", ctypes.c_float * 12)]


class lidar_beams(ctypes.Structure):
    _fields_ = [(n, c_vp) for n in ("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst", "sub",
                                    "theta_deg", "rf")]


class lidar_points(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64)] + [(n, c_vp) for n in ("xyz", "range", "intensity", "normal",
                                                                      "material", "instance", "beam", "frame")]


class lidar_work_counts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("rays", "node_bytes", "node_visits", "tri_tests", "unique_nodes",
                                               "unique_tris")]


class lidar_launch_config(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("tile_rays", ctypes.c_int32), ("ray_order", ctypes.c_int32), ("traversal", ctypes.c_int32),
                ("fused_scatter", ctypes.c_int32)]


class lidar_sweep_frame(ctypes.Structure):
    _fields_ = [("sensor", ctypes.c_int32), ("frame", ctypes.c_int32), ("pose0", ctypes.c_float * 12),
                ("pose1", ctypes.c_float * 12)]


class lidar_echoes(ctypes.Structure):
    _fields_ = [("n_echoes", ctypes.c_int32), ("mode", ctypes.c_int32), ("separation", ctypes.c_float)] + \
               [(n, c_vp) for n in ("count", "range", "intensity", "tri", "sub")]


class lidar_build_options(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("ploc_radius", ctypes.c_int32), ("collapse", ctypes.c_int32),
                ("tri_cost", ctypes.c_float), ("treelet_rounds", ctypes.c_int32),
                ("area_weight", ctypes.c_float * 3)]


class lidar_raster_config(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("n_cameras", ctypes.c_int32)]


assert ctypes.sizeof(lidar_frame) == 56
assert ctypes.sizeof(lidar_sweep_frame) == 104

_lock = threading.Lock()
_lib = None

# (name, restype, argtypes); restype None means lidar_status checked by _call
_PROTOS = [
    ("lidar_create", ctypes.c_int, [ctypes.c_int, c_vp, ctypes.POINTER(c_vp)]),
    ("lidar_destroy", None, [c_vp]),
    ("lidar_last_error", ctypes.c_char_p, []),
    ("lidar_sync_status", ctypes.c_int, [c_vp]),
    ("lidar_scene_build", ctypes.c_int, [c_vp, c_vp, ctypes.c_int64, c_vp, ctypes.c_int64, c_vp, c_vp,
                                         ctypes.POINTER(c_vp)]),
    ("lidar_scene_free", None, [c_vp]),
    ("lidar_get_scene_info", ctypes.c_int, [c_vp, ctypes.POINTER(lidar_scene_info)]),
    ("lidar_scene_export", ctypes.c_int, [c_vp, c_vp, c_vp]),
    ("lidar_scene_export_wide", ctypes.c_int, [c_vp, ctypes.c_int32, c_vp]),
    ("lidar_set_sensor", ctypes.c_int, [c_vp, ctypes.c_int32, ctypes.POINTER(lidar_sensor_desc)]),
    ("lidar_set_sensor_gain", ctypes.c_int, [c_vp, ctypes.c_int32, ctypes.c_float]),
    ("lidar_get_beam_dirs", ctypes.c_int, [c_vp, ctypes.c_int32, c_vp]),
    ("lidar_build_tables", ctypes.c_int, [c_vp, c_vp, ctypes.c_int32, c_vp]),
    ("lidar_build_tables_backward", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int32, c_vp]),
    ("lidar_set_materials", ctypes.c_int, [c_vp, c_vp, ctypes.c_int32]),
    ("lidar_cast", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int32, ctypes.c_uint64,
                                  ctypes.POINTER(lidar_beams), ctypes.POINTER(lidar_points), c_vp]),
    ("lidar_points_download", ctypes.c_int, [c_vp, ctypes.POINTER(lidar_points), ctypes.POINTER(lidar_points),
                                             ctypes.c_int64, c_vp]),
    ("lidar_batch_create", ctypes.c_int, [c_vp, c_vp, ctypes.c_int32, ctypes.POINTER(c_vp)]),
    ("lidar_batch_free", None, [c_vp]),
    ("lidar_batch_set_poses", ctypes.c_int, [c_vp, c_vp, c_vp]),
    ("lidar_cast_batch", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_uint64, ctypes.POINTER(lidar_beams),
                                        ctypes.POINTER(lidar_points), c_vp]),
    ("lidar_graph_create", ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, ctypes.c_uint64, ctypes.POINTER(lidar_beams),
                                          ctypes.POINTER(lidar_points), c_vp, ctypes.POINTER(c_vp)]),
    ("lidar_graph_launch", ctypes.c_int, [c_vp]),
    ("lidar_graph_free", None, [c_vp]),
    ("lidar_cast_backward", ctypes.c_int, [c_vp, ctypes.c_int64, ctypes.POINTER(lidar_beams), ctypes.c_float,
                                           c_vp, c_vp, c_vp]),
    ("lidar_cast_backward_mse", ctypes.c_int, [c_vp, ctypes.c_int64, ctypes.POINTER(lidar_beams),
                                               ctypes.c_float, c_vp, c_vp, c_vp, c_vp, c_vp]),
    ("lidar_cast_backward_mse_count", ctypes.c_int, [c_vp, ctypes.c_int64, ctypes.POINTER(lidar_beams),
                                                     ctypes.c_float, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    ("lidar_cast_backward_mse_noalloc", ctypes.c_int, [c_vp, ctypes.c_int64, c_vp, c_vp, c_vp, c_vp, c_vp,
                                                       ctypes.c_int32, ctypes.c_float, c_vp, c_vp, c_vp, c_vp,
                                                       c_vp]),
    ("lidar_count_work", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.POINTER(lidar_work_counts), c_vp]),
    ("lidar_schedule_by_cost", ctypes.c_int, [c_vp, c_vp, ctypes.POINTER(lidar_frame), ctypes.c_uint64,
                                              ctypes.c_int32]),
    ("lidar_reset_schedule", ctypes.c_int, [c_vp, ctypes.c_int32]),
    ("lidar_cast_sweep", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.POINTER(lidar_beams), ctypes.POINTER(lidar_echoes)]),
    ("lidar_raster_cast", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int32, ctypes.c_uint64,
                                         ctypes.POINTER(lidar_raster_config), ctypes.POINTER(lidar_beams)]),
    ("lidar_raster_gbuffer", ctypes.c_int, [c_vp, c_vp, ctypes.POINTER(lidar_frame),
                                            ctypes.POINTER(lidar_raster_config), c_vp, c_vp, c_vp, c_vp]),
    ("lidar_set_build_options", ctypes.c_int, [c_vp, ctypes.POINTER(lidar_build_options)]),
    ("lidar_get_build_options", ctypes.c_int, [c_vp, ctypes.POINTER(lidar_build_options)]),
    ("lidar_get_launch_config", ctypes.c_int, [c_vp, ctypes.POINTER(lidar_launch_config)]),
    ("lidar_set_launch_config", ctypes.c_int, [c_vp, ctypes.POINTER(lidar_launch_config)]),
    ("lidar_set_wait_limit", ctypes.c_int, [c_vp, ctypes.c_uint64]),
    ("lidar_set_cast_overlap", ctypes.c_int, [c_vp, ctypes.c_int32]),
    ("lidar_get_cast_overlap", ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_int32)]),
    ("lidar_measure_fp32_rate", ctypes.c_int, [c_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    ("lidar_get_wait_limit", ctypes.c_int, [c_vp, ctypes.POINTER(ctypes.c_uint64)]),
]

EXPORTED = [p[0] for p in _PROTOS]


def load(path: str = None):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
            L = ctypes.CDLL(p)
            for name, res, args in _PROTOS:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return load().lidar_last_error().decode(errors="replace")


def check(status: int, what: str = ""):
    if status != LIDAR_OK:
        raise LidarError(status, f"{what}: {last_error()}")
    return status


def _fwd(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    return f


lidar_create = _fwd("lidar_create")
lidar_destroy = _fwd("lidar_destroy")
lidar_last_error = _fwd("lidar_last_error")
lidar_sync_status = _fwd("lidar_sync_status")
lidar_scene_build = _fwd("lidar_scene_build")
lidar_scene_free = _fwd("lidar_scene_free")
lidar_get_scene_info = _fwd("lidar_get_scene_info")
lidar_scene_export = _fwd("lidar_scene_export")
lidar_scene_export_wide = _fwd("lidar_scene_export_wide")
lidar_set_sensor = _fwd("lidar_set_sensor")
lidar_set_sensor_gain = _fwd("lidar_set_sensor_gain")
lidar_get_beam_dirs = _fwd("lidar_get_beam_dirs")
lidar_build_tables = _fwd("lidar_build_tables")
lidar_build_tables_backward = _fwd("lidar_build_tables_backward")
lidar_set_materials = _fwd("lidar_set_materials")
lidar_cast = _fwd("lidar_cast")
lidar_points_download = _fwd("lidar_points_download")
lidar_batch_create = _fwd("lidar_batch_create")
lidar_batch_free = _fwd("lidar_batch_free")
lidar_batch_set_poses = _fwd("lidar_batch_set_poses")
lidar_cast_batch = _fwd("lidar_cast_batch")
lidar_graph_create = _fwd("lidar_graph_create")
lidar_graph_launch = _fwd("lidar_graph_launch")
lidar_graph_free = _fwd("lidar_graph_free")
lidar_cast_backward = _fwd("lidar_cast_backward")
lidar_cast_backward_mse = _fwd("lidar_cast_backward_mse")
lidar_cast_backward_mse_count = _fwd("lidar_cast_backward_mse_count")
lidar_cast_backward_mse_noalloc = _fwd("lidar_cast_backward_mse_noalloc")
lidar_count_work = _fwd("lidar_count_work")
lidar_raster_cast = _fwd("lidar_raster_cast")
lidar_cast_sweep = _fwd("lidar_cast_sweep")
lidar_set_build_options = _fwd("lidar_set_build_options")
lidar_get_build_options = _fwd("lidar_get_build_options")
lidar_raster_gbuffer = _fwd("lidar_raster_gbuffer")
lidar_schedule_by_cost = _fwd("lidar_schedule_by_cost")
lidar_reset_schedule = _fwd("lidar_reset_schedule")
lidar_get_launch_config = _fwd("lidar_get_launch_config")
lidar_set_launch_config = _fwd("lidar_set_launch_config")
lidar_set_wait_limit = _fwd("lidar_set_wait_limit")
lidar_get_wait_limit = _fwd("lidar_get_wait_limit")
lidar_measure_fp32_rate = _fwd("lidar_measure_fp32_rate")
lidar_set_cast_overlap = _fwd("lidar_set_cast_overlap")
lidar_get_cast_overlap = _fwd("lidar_get_cast_overlap")
