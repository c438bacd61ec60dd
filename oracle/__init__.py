"""ORACLE — test infrastructure only.

ctypes wrapper around ``lidar_oracle.c``, the plain FP64 CPU implementation of
per-beam LiDAR return generation.  Only the tests, the package smoke check and
the benchmark's CPU-baseline leg may import this package; the product path
never does, and this package imports nothing from the product package.

Pins (tests/test_oracle_*.py) tie every function here to something other than
itself: closed forms on planes, exact-rational brute force on tiny scenes,
numpy's Philox, finite differences, and invariants under rigid motion and
triangle permutation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lidar_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NO_HIT = 0xFFFFFFFF
NTAB = 91
FLAG_EDGE, FLAG_TIE, FLAG_CUTOFF, FLAG_SUBTIE, FLAG_GRAZING = 1, 2, 4, 8, 16


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Sensor(ctypes.Structure):
    _fields_ = [("n_beams", ctypes.c_int64), ("az", ctypes.c_void_p), ("el", ctypes.c_void_p),
                ("r_min", ctypes.c_float), ("r_max", ctypes.c_float), ("d_max", ctypes.c_float),
                ("RL_max", ctypes.c_float), ("sigma", ctypes.c_float), ("gain", ctypes.c_float),
                ("range_exp", ctypes.c_float), ("r_ref", ctypes.c_float), ("divergence", ctypes.c_float),
                ("n_sub", ctypes.c_int32), ("sigma_k", ctypes.c_float)]


class _Out(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("valid", "tri", "t", "range", "intensity", "normal", "xyz", "mat", "inst", "theta_deg",
                 "R", "rf", "sub", "flags", "sub_valid", "sub_I", "sub_range", "sub_tri", "sub_flags")]


class _RasterCfg(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("n_cameras", ctypes.c_int32)]


class _RasterOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("valid", "outside", "cam", "px", "py", "tri", "q_depth", "q_angle", "mat", "inst", "t", "z",
                 "range", "intensity", "theta_deg", "flags")]


class _Echoes(ctypes.Structure):
    _fields_ = [("n_echoes", ctypes.c_int32), ("mode", ctypes.c_int32), ("separation", ctypes.c_float)] + \
               [(n, ctypes.c_void_p) for n in ("count", "range", "intensity", "tri", "sub")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
            L.oracle_beam_dirs.argtypes = [i64, vp, vp, vp]
            L.oracle_subray_offsets.argtypes = [ctypes.c_float, i32, vp, vp]
            L.oracle_world_ray.argtypes = [vp, vp, vp, vp]
            L.oracle_subray_dir.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_int, vp]
            L.oracle_philox4x64_10.argtypes = [vp, vp, vp]
            L.oracle_normal.argtypes = [u64, u64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            L.oracle_normal.restype = ctypes.c_double
            L.oracle_build_tables.argtypes = [vp, i32, vp]
            L.oracle_build_tables_backward.argtypes = [vp, vp, i32, vp]
            L.oracle_cast.argtypes = [vp, i64, vp, i64, vp, vp, vp, i32, vp, i32, vp, i32, u64, vp, vp, i64,
                                      i32, ctypes.POINTER(_Out), i32]
            L.oracle_cast.restype = ctypes.c_int
            L.oracle_loss.argtypes = [i64, vp, vp, vp, vp, vp, i32, ctypes.c_double, vp, vp]
            L.oracle_loss.restype = ctypes.c_double
            L.oracle_cast_backward.argtypes = [i64, vp, vp, vp, vp, vp, i32, ctypes.c_double, vp, vp, vp,
                                               vp, vp]
            L.oracle_cast_backward.restype = i64
            L.oracle_max_threads.restype = i32
            L.oracle_raster.argtypes = [vp, i64, vp, i64, vp, vp, vp, i32, vp, i32, vp, i32, u64,
                                        ctypes.POINTER(_RasterCfg), vp, vp, i64, ctypes.POINTER(_RasterOut), i32]
            L.oracle_raster.restype = ctypes.c_int
            L.oracle_raster_constants.argtypes = [i32, i32, vp, vp, vp, vp]
            L.oracle_sweep_fraction.argtypes = [ctypes.c_double]
            L.oracle_sweep_fraction.restype = ctypes.c_float
            L.oracle_sweep_quaternions.argtypes = [vp, vp, vp, vp]
            L.oracle_sweep_pose.argtypes = [vp, vp, vp, vp, ctypes.c_float, vp]
            L.oracle_cast_sweep.argtypes = [vp, i64, vp, i64, vp, vp, vp, i32, vp, i32, vp, i32, u64, vp, vp, i64,
                                            i32, ctypes.POINTER(_Out), ctypes.POINTER(_Echoes), i32]
            L.oracle_cast_sweep.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ pieces

def beam_dirs(az, el):
    az = _c(az, np.float64)
    el = _c(el, np.float64)
    out = np.empty((az.size, 3), np.float32)
    lib().oracle_beam_dirs(az.size, _p(az), _p(el), _p(out))
    return out


def subray_offsets(divergence, n_sub):
    a = np.zeros(max(n_sub, 1), np.float32)
    b = np.zeros(max(n_sub, 1), np.float32)
    lib().oracle_subray_offsets(ctypes.c_float(divergence), n_sub, _p(a), _p(b))
    return a, b


def world_ray(pose12, d):
    pose12 = _c(pose12, np.float32)
    d = _c(d, np.float32)
    o = np.empty(3, np.float32)
    w = np.empty(3, np.float32)
    lib().oracle_world_ray(_p(pose12), _p(d), _p(o), _p(w))
    return o, w


def subray_dir(d, alpha, beta, k):
    d = _c(d, np.float32)
    out = np.empty(3, np.float32)
    lib().oracle_subray_dir(_p(d), ctypes.c_float(alpha), ctypes.c_float(beta), k, _p(out))
    return out


def philox4x64_10(ctr, key):
    ctr = _c(ctr, np.uint64)
    key = _c(key, np.uint64)
    out = np.empty(4, np.uint64)
    lib().oracle_philox4x64_10(_p(ctr), _p(key), _p(out))
    return out


def normal(seed, beam, frame, sensor, sub):
    return lib().oracle_normal(seed, beam, frame, sensor, sub)


def build_tables(params):
    params = _c(params, np.float32).reshape(-1, 3)
    out = np.empty((params.shape[0], NTAB), np.float64)
    lib().oracle_build_tables(_p(params), params.shape[0], _p(out))
    return out


def build_tables_backward(params, grad_table):
    params = _c(params, np.float32).reshape(-1, 3)
    grad_table = _c(grad_table, np.float64)
    out = np.empty((params.shape[0], 3), np.float64)
    lib().oracle_build_tables_backward(_p(params), _p(grad_table), params.shape[0], _p(out))
    return out


def max_threads():
    return lib().oracle_max_threads()


# ------------------------------------------------------------------ cast

class CastResult(dict):
    """Per-sample oracle outputs (numpy arrays keyed by name)."""

    def __getattr__(self, k):
        return self[k]


def _inputs(scene, sensors, frames, table, samples):
    verts = _c(scene.verts, np.float32)
    tris = _c(scene.tris, np.uint32)
    mat = _c(scene.mat, np.uint16)
    inst = _c(scene.inst, np.uint32)
    table = _c(table, np.float64)
    keep = []
    sens = (_Sensor * len(sensors))()
    for i, s in enumerate(sensors):
        az = _c(s.az_rad, np.float64)
        el = _c(s.el_rad, np.float64)
        keep += [az, el]
        sens[i] = _Sensor(az.size, az.ctypes.data, el.ctypes.data, s.r_min, s.r_max, s.d_max, s.RL_max,
                          s.sigma, s.gain, s.range_exp, s.r_ref, s.divergence_rad, s.n_subrays,
                          getattr(s, "sigma_k", 0.0))
    fr = np.ascontiguousarray(frames)
    assert fr.dtype.itemsize == 56
    if samples is None:
        sf, sb = [], []
        for k, f in enumerate(fr):
            nb = sensors[int(f["sensor"])].n_beams
            sf.append(np.full(nb, k, np.int64))
            sb.append(np.arange(nb, dtype=np.int64))
        sf = np.concatenate(sf)
        sb = np.concatenate(sb)
    else:
        sf = _c(samples[0], np.int64)
        sb = _c(samples[1], np.int64)
    return verts, tris, mat, inst, table, sens, keep, fr, sf, sb


def raster_constants(width, n_cameras):
    """(f, c, cos[K], sin[K]) of the raster path's cameras, FP32."""
    f = np.zeros(1, np.float32)
    c = np.zeros(1, np.float32)
    ck = np.zeros(n_cameras, np.float32)
    sk = np.zeros(n_cameras, np.float32)
    lib().oracle_raster_constants(width, n_cameras, _p(f), _p(c), _p(ck), _p(sk))
    return float(f[0]), float(c[0]), ck, sk


def raster(scene, sensors, frames, table, seed, width, n_cameras, samples=None, n_threads=0):
    """The raster-and-resample path (K pin-hole cameras of W x W pixels per
    frame, 24-bit depth and angle, 8-bit material, 24-bit instance, each beam
    reading its pixel) on (frame entry, beam) samples."""
    verts, tris, mat, inst, table, sens, keep, fr, sf, sb = _inputs(scene, sensors, frames, table, samples)
    n = sf.size
    R = CastResult(
        valid=np.zeros(n, np.uint8), outside=np.zeros(n, np.uint8), cam=np.zeros(n, np.int32),
        px=np.zeros(n, np.int32), py=np.zeros(n, np.int32), tri=np.zeros(n, np.uint32),
        q_depth=np.zeros(n, np.uint32), q_angle=np.zeros(n, np.uint32), mat=np.zeros(n, np.uint16),
        inst=np.zeros(n, np.uint32), t=np.zeros(n), z=np.zeros(n), range=np.zeros(n), intensity=np.zeros(n),
        theta_deg=np.zeros(n), flags=np.zeros(n, np.uint32), sample_frame=sf, sample_beam=sb)
    out = _RasterOut(*[R[name].ctypes.data for name, _ in _RasterOut._fields_])
    cfg = _RasterCfg(width, n_cameras)
    rc = lib().oracle_raster(_p(verts), verts.shape[0], _p(tris), tris.shape[0], _p(mat), _p(inst), sens,
                             len(sensors), fr.ctypes.data_as(ctypes.c_void_p), len(fr), _p(table),
                             table.shape[0], seed, ctypes.byref(cfg), _p(sf), _p(sb), n, ctypes.byref(out),
                             n_threads)
    if rc != 0:
        raise ValueError("oracle_raster rejected its inputs")
    return R


def sweep_fraction(az):
    return float(lib().oracle_sweep_fraction(float(az)))


def sweep_quaternions(pose0, pose1):
    p0 = _c(pose0, np.float32).reshape(12)
    p1 = _c(pose1, np.float32).reshape(12)
    q0 = np.zeros(4, np.float32)
    q1 = np.zeros(4, np.float32)
    lib().oracle_sweep_quaternions(_p(p0), _p(p1), _p(q0), _p(q1))
    return q0, q1


def sweep_pose(pose0, pose1, s):
    """Pose (row-major 3x4, FP32) at fraction s of a sweep from pose0 to pose1."""
    p0 = _c(pose0, np.float32).reshape(12)
    p1 = _c(pose1, np.float32).reshape(12)
    q0, q1 = sweep_quaternions(p0, p1)
    P = np.zeros(12, np.float32)
    lib().oracle_sweep_pose(_p(q0), _p(q1), _p(p0), _p(p1), float(s), _p(P))
    return P


def cast_sweep(scene, sensors, frames, table, seed, samples=None, echoes=None, n_threads=0):
    """Rolling-shutter cast: `frames` has SWEEP_FRAME_DTYPE (pose0 at the
    sweep's start, pose1 at its end); each beam sees the pose at its firing
    fraction.  `echoes` = (n_echoes, mode, separation) adds the multi-echo
    outputs echo_count, echo_range, echo_intensity, echo_tri, echo_sub."""
    fr = np.ascontiguousarray(frames)
    assert fr.dtype.itemsize == 104
    if samples is None:
        sf, sb = [], []
        for k, f in enumerate(fr):
            nb = sensors[int(f["sensor"])].n_beams
            sf.append(np.full(nb, k, np.int64))
            sb.append(np.arange(nb, dtype=np.int64))
        samples = (np.concatenate(sf), np.concatenate(sb))
    verts, tris, mat, inst, table, sens, keep, _, sf, sb = _inputs(scene, sensors, np.zeros(0, dtype=[
        ("sensor", np.int32), ("frame", np.int32), ("pose", np.float32, (12,))]), table, samples)
    n = sf.size
    nsub = max(int(s.n_subrays) for s in sensors)
    R = CastResult(
        valid=np.zeros(n, np.uint8), tri=np.zeros(n, np.uint32), t=np.zeros(n), range=np.zeros(n),
        intensity=np.zeros(n), normal=np.zeros((n, 3)), xyz=np.zeros((n, 3)), mat=np.zeros(n, np.uint16),
        inst=np.zeros(n, np.uint32), theta_deg=np.zeros(n), R=np.zeros(n), rf=np.zeros(n),
        sub=np.zeros(n, np.int32), flags=np.zeros(n, np.uint32),
        sub_valid=np.zeros((n, nsub), np.uint8), sub_I=np.zeros((n, nsub)), sub_range=np.zeros((n, nsub)),
        sub_tri=np.zeros((n, nsub), np.uint32), sub_flags=np.zeros((n, nsub), np.uint32),
        sample_frame=sf, sample_beam=sb)
    out = _Out(*[R[name].ctypes.data for name, _ in _Out._fields_])
    ep = None
    if echoes is not None:
        ne, mode, sep = echoes
        R.update(echo_count=np.zeros(n, np.uint8), echo_range=np.zeros((n, ne)), echo_intensity=np.zeros((n, ne)),
                 echo_tri=np.zeros((n, ne), np.uint32), echo_sub=np.zeros((n, ne), np.int32))
        ep = _Echoes(ne, mode, sep, R["echo_count"].ctypes.data, R["echo_range"].ctypes.data,
                     R["echo_intensity"].ctypes.data, R["echo_tri"].ctypes.data, R["echo_sub"].ctypes.data)
    rc = lib().oracle_cast_sweep(_p(verts), verts.shape[0], _p(tris), tris.shape[0], _p(mat), _p(inst), sens,
                                 len(sensors), fr.ctypes.data_as(ctypes.c_void_p), len(fr), _p(table),
                                 table.shape[0], seed, _p(sf), _p(sb), n, nsub, ctypes.byref(out),
                                 ctypes.byref(ep) if ep is not None else None, n_threads)
    if rc != 0:
        raise ValueError("oracle_cast_sweep rejected its inputs")
    return R


def cast(scene, sensors, frames, table, seed, samples=None, n_threads=0):
    """Run the oracle on (frame entry, beam) samples (default: every beam of
    every frame).  `scene` has verts/tris/mat/inst; `sensors` are objects with
    the SensorSpec fields; `frames` is a structured array (sensor, frame,
    pose[12]); `table` is [M][91] FP64."""
    verts = _c(scene.verts, np.float32)
    tris = _c(scene.tris, np.uint32)
    mat = _c(scene.mat, np.uint16)
    inst = _c(scene.inst, np.uint32)
    table = _c(table, np.float64)
    keep = []
    sens = (_Sensor * len(sensors))()
    for i, s in enumerate(sensors):
        az = _c(s.az_rad, np.float64)
        el = _c(s.el_rad, np.float64)
        keep += [az, el]
        sens[i] = _Sensor(az.size, az.ctypes.data, el.ctypes.data, s.r_min, s.r_max, s.d_max, s.RL_max,
                          s.sigma, s.gain, s.range_exp, s.r_ref, s.divergence_rad, s.n_subrays,
                          getattr(s, "sigma_k", 0.0))
    fr = np.ascontiguousarray(frames)
    assert fr.dtype.itemsize == 56
    if samples is None:
        sf, sb = [], []
        for k, f in enumerate(fr):
            nb = sensors[int(f["sensor"])].n_beams
            sf.append(np.full(nb, k, np.int64))
            sb.append(np.arange(nb, dtype=np.int64))
        sf = np.concatenate(sf)
        sb = np.concatenate(sb)
    else:
        sf = _c(samples[0], np.int64)
        sb = _c(samples[1], np.int64)
    n = sf.size
    nsub = max(int(s.n_subrays) for s in sensors)
    R = CastResult(
        valid=np.zeros(n, np.uint8), tri=np.zeros(n, np.uint32), t=np.zeros(n), range=np.zeros(n),
        intensity=np.zeros(n), normal=np.zeros((n, 3)), xyz=np.zeros((n, 3)), mat=np.zeros(n, np.uint16),
        inst=np.zeros(n, np.uint32), theta_deg=np.zeros(n), R=np.zeros(n), rf=np.zeros(n),
        sub=np.zeros(n, np.int32), flags=np.zeros(n, np.uint32),
        sub_valid=np.zeros((n, nsub), np.uint8), sub_I=np.zeros((n, nsub)), sub_range=np.zeros((n, nsub)),
        sub_tri=np.zeros((n, nsub), np.uint32), sub_flags=np.zeros((n, nsub), np.uint32),
        sample_frame=sf, sample_beam=sb)
    out = _Out(*[R[name].ctypes.data for name, _ in _Out._fields_])
    rc = lib().oracle_cast(_p(verts), verts.shape[0], _p(tris), tris.shape[0], _p(mat), _p(inst), sens,
                           len(sensors), fr.ctypes.data_as(ctypes.c_void_p), len(fr), _p(table),
                           table.shape[0], seed, _p(sf), _p(sb), n, nsub, ctypes.byref(out), n_threads)
    if rc != 0:
        raise ValueError("oracle_cast rejected its inputs")
    return R


def loss(valid, mat, theta_deg, rf, table, gain, target_I, target_valid):
    a = [_c(valid, np.uint8), _c(mat, np.uint16), _c(theta_deg, np.float64), _c(rf, np.float64)]
    table = _c(table, np.float64)
    tI = _c(target_I, np.float64)
    tv = _c(target_valid, np.uint8)
    return lib().oracle_loss(a[0].size, *[_p(x) for x in a], _p(table), table.shape[0], gain, _p(tI), _p(tv))


def cast_backward(valid, mat, theta_deg, rf, table, gain, target_I, target_valid):
    """Returns (loss, dL/dT [M][91], dL/dg, N)."""
    a = [_c(valid, np.uint8), _c(mat, np.uint16), _c(theta_deg, np.float64), _c(rf, np.float64)]
    table = _c(table, np.float64)
    tI = _c(target_I, np.float64)
    tv = _c(target_valid, np.uint8)
    gt = np.zeros_like(table)
    L = np.zeros(1)
    gg = np.zeros(1)
    N = lib().oracle_cast_backward(a[0].size, *[_p(x) for x in a], _p(table), table.shape[0], gain, _p(tI),
                                   _p(tv), _p(L), _p(gt), _p(gg))
    return float(L[0]), gt, float(gg[0]), int(N)
