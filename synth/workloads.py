"""The five benchmark workloads plus small variants, all seeded.

Seeds: scene = 1000 + cfg, noise = 2000 + cfg, trajectory = 3000 + cfg,
hidden reflectance parameters (differentiation workload) = 4000.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from . import geometry as G
from . import sensors as S

SEED_SCENE = 1000
SEED_NOISE = 2000
SEED_TRAJ = 3000
SEED_HIDDEN = 4000

FRAME_DTYPE = np.dtype([("sensor", np.int32), ("frame", np.int32), ("pose", np.float32, (12,))],
                       align=False)


@dataclasses.dataclass
class Scene:
    verts: np.ndarray   # float32 [V,3]
    tris: np.ndarray    # uint32  [T,3]
    mat: np.ndarray     # uint16  [T]
    inst: np.ndarray    # uint32  [T]

    @property
    def n_tris(self):
        return int(self.tris.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    sensors: List[S.SensorSpec]
    frames: np.ndarray          # FRAME_DTYPE [F]
    params: np.ndarray          # float32 [M,3] (a, s, w_deg)
    seed: int                   # noise key
    hidden_params: np.ndarray = None   # differentiation target, float32 [M,3]

    @property
    def n_rays(self):
        return int(sum(self.sensors[f["sensor"]].n_beams * self.sensors[f["sensor"]].n_subrays
                       for f in self.frames))

    @property
    def n_beams_total(self):
        return int(sum(self.sensors[f["sensor"]].n_beams for f in self.frames))


def pose_rows(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Row-major 3x4 [R | t] (sensor -> world), rounded once to float32."""
    P = np.concatenate([np.asarray(R, np.float64), np.asarray(t, np.float64).reshape(3, 1)], axis=1)
    return P.reshape(12).astype(np.float32)


# a sweep: the pose at its start and at its end (rolling shutter)
SWEEP_FRAME_DTYPE = np.dtype([("sensor", np.int32), ("frame", np.int32), ("pose0", np.float32, (12,)),
                              ("pose1", np.float32, (12,))], align=False)


def make_sweep_frames(entries):
    """entries: (sensor, frame, pose0 rows [12], pose1 rows [12])."""
    fr = np.zeros(len(entries), dtype=SWEEP_FRAME_DTYPE)
    for i, (s, f, p0, p1) in enumerate(entries):
        fr[i]["sensor"] = s
        fr[i]["frame"] = f
        fr[i]["pose0"] = np.asarray(p0, np.float32).reshape(12)
        fr[i]["pose1"] = np.asarray(p1, np.float32).reshape(12)
    return fr


def make_frames(entries):
    fr = np.zeros(len(entries), dtype=FRAME_DTYPE)
    for k, (s, f, pose) in enumerate(entries):
        fr[k]["sensor"] = s
        fr[k]["frame"] = f
        fr[k]["pose"] = pose
    return fr


# ------------------------------------------------------------------- cfg 0

def ground_boxes_scene(rng, n_boxes=64, half=100.0, n_materials=4, sensor_xy=(0.0, 0.0),
                       clearance=3.0):
    mb = G.MeshBuilder()
    q = np.array([[-half, -half, 0.0], [half, -half, 0.0], [half, half, 0.0], [-half, half, 0.0]])
    mb.add(q, [[0, 1, 2], [0, 2, 3]], 0, 0)
    bv, bt = G.unit_box_faces(1)
    k = 0
    while k < n_boxes:
        side = rng.uniform(1.0, 10.0, size=3)
        c = rng.uniform(-(half - 5.0), half - 5.0, size=2)
        lo = c - side[:2] / 2
        hi = c + side[:2] / 2
        d = np.maximum(np.maximum(lo - sensor_xy, np.asarray(sensor_xy) - hi), 0.0)
        if np.hypot(d[0], d[1]) < clearance:
            continue
        m = int(rng.integers(0, n_materials))
        v = bv * side + np.array([c[0], c[1], side[2] / 2])
        mb.add(v, bt, m, 1 + k)
        k += 1
    return Scene(*mb.build())


def cfg0():
    rng = np.random.default_rng(SEED_SCENE + 0)
    scene = ground_boxes_scene(rng)
    params = S.material_params(np.random.default_rng((SEED_SCENE + 0, 1)), 4)
    sensor = S.sensor_16ch(1800, r_min=0.5, r_max=100.0, d_max=100.0, RL_max=0.8, sigma=0.02)
    frames = make_frames([(0, 0, pose_rows(np.eye(3), [0.0, 0.0, 1.8]))])
    return Workload("cfg0_16ch_770tri", scene, [sensor], frames, params, SEED_NOISE + 0)


# ------------------------------------------------------------------- cfg 1

def trajectory(rng, n_frames, dt=0.1, amp_max=80.0, f_max=0.05):
    """Smooth random path: x(t), y(t) each a sum of 3 sinusoids with total
    amplitude <= amp_max and frequencies <= f_max; yaw follows the heading."""
    t = np.arange(n_frames) * dt
    out = []
    for _axis in range(2):
        A = rng.uniform(0.2, 1.0, size=3)
        A = A / A.sum() * rng.uniform(0.5, 1.0) * amp_max
        f = rng.uniform(0.2 * f_max, f_max, size=3)
        ph = rng.uniform(0.0, 2 * np.pi, size=3)
        p = sum(A[k] * np.sin(2 * np.pi * f[k] * t + ph[k]) for k in range(3))
        dp = sum(A[k] * 2 * np.pi * f[k] * np.cos(2 * np.pi * f[k] * t + ph[k]) for k in range(3))
        # start the path at the origin
        p = p - A @ np.sin(ph)
        out.append((p, dp))
    (x, dx), (y, dy) = out
    yaw = np.arctan2(dy, dx)
    return x, y, yaw


def terrain_objects_scene(rng, n_cells=512, half=256.0, n_objects=2000, obj_half=250.0,
                          n_materials=32, keepout=None, keepout_r=8.0, amplitude=5.0):
    fbm = G.ValueNoiseFBM(rng, half, amplitude=amplitude)
    mb = G.MeshBuilder()
    tv, tt, (ix, iy) = G.grid_terrain(n_cells, half, fbm)
    # terrain materials 0..3 on a 64 m random patchwork
    patch = rng.integers(0, 4, size=(n_cells // 64 + 1, n_cells // 64 + 1))
    cell_scale = 2 * half / n_cells
    px = np.minimum((ix * cell_scale / 64.0).astype(np.int64), patch.shape[1] - 1)
    py = np.minimum((iy * cell_scale / 64.0).astype(np.int64), patch.shape[0] - 1)
    tmat = np.repeat(patch[py, px], 2).astype(np.uint16)
    mb.add(tv, tt, tmat, 0)
    bv, bt = G.unit_box_faces(4)
    sv, st = G.icosphere(2)
    k = 0
    while k < n_objects:
        c = rng.uniform(-obj_half, obj_half, size=2)
        if keepout is not None and np.min(np.hypot(keepout[:, 0] - c[0], keepout[:, 1] - c[1])) < keepout_r:
            continue
        h = float(fbm(c[0], c[1]))
        m = int(rng.integers(4, n_materials))
        yaw = rng.uniform(0, 2 * np.pi)
        if k % 2 == 0:
            side = rng.uniform(0.5, 6.0, size=3)
            v = (bv * side) @ G.rot_z(yaw).T + np.array([c[0], c[1], h + side[2] / 2 - 0.2])
            mb.add(v, bt, m, 1 + k)
        else:
            r = rng.uniform(0.3, 3.0)
            v = (sv * r) @ G.rot_z(yaw).T + np.array([c[0], c[1], h + 0.8 * r])
            mb.add(v, st, m, 1 + k)
        k += 1
    return Scene(*mb.build()), fbm


# vehicle-frame mounts for the 8-sensor rig: (sensor kind, offset, yaw deg, pitch deg)
RIG = [
    ("spin16", (2.0, 1.0, -0.3), 45.0, 0.0),
    ("spin16", (2.0, -1.0, -0.3), -45.0, 0.0),
    ("spin32", (-2.0, 1.0, -0.3), 135.0, 0.0),
    ("spin32", (-2.0, -1.0, -0.3), -135.0, 0.0),
    ("spin64", (0.0, 1.0, 0.2), 90.0, 0.0),
    ("spin64", (0.0, -1.0, 0.2), -90.0, 0.0),
    ("spin128", (0.0, 0.0, 0.0), 0.0, 0.0),
    ("raster", (2.2, 0.0, -0.5), 0.0, -5.0),
]


def _rig_sensor(kind):
    if kind == "spin16":
        return S.sensor_16ch(1800, r_min=0.5, r_max=100.0, d_max=100.0)
    if kind == "spin32":
        return S.sensor_32ch(2048, r_min=0.5, r_max=200.0, d_max=200.0)
    if kind == "spin64":
        return S.sensor_64ch(2048, r_min=0.5, r_max=200.0, d_max=200.0)
    if kind == "spin128":
        return S.sensor_128ch(2048, r_min=0.5, r_max=200.0, d_max=200.0)
    return S.sensor_raster(256, 128, 120.0, 25.0, r_min=0.5, r_max=200.0, d_max=200.0)


_CFG1_CACHE = {}


def _cfg1_scene():
    """The 1M-triangle terrain + objects scene shared by cfg1, cfg2 and cfg3.
    Objects keep clear of the trajectory the batched workloads drive along."""
    if "scene" not in _CFG1_CACHE:
        tx, ty, _ = trajectory(np.random.default_rng(SEED_TRAJ + 2), 64)
        keep = np.concatenate([np.stack([tx, ty], 1), [[0.0, 0.0]]], 0)
        rng = np.random.default_rng(SEED_SCENE + 1)
        scene, fbm = terrain_objects_scene(rng, keepout=keep)
        _CFG1_CACHE["scene"] = (scene, fbm)
    return _CFG1_CACHE["scene"]


def cfg1():
    scene, fbm = _cfg1_scene()
    params = S.material_params(np.random.default_rng((SEED_SCENE + 1, 1)), 32)
    sensor = S.sensor_128ch(2048, r_min=0.5, r_max=200.0, d_max=200.0)
    z = float(fbm(0.0, 0.0)) + 2.0
    frames = make_frames([(0, 0, pose_rows(np.eye(3), [0.0, 0.0, z]))])
    return Workload("cfg1_128ch_1Mtri", scene, [sensor], frames, params, SEED_NOISE + 1)


def vehicle_poses(fbm, n_frames, traj_seed):
    x, y, yaw = trajectory(np.random.default_rng(traj_seed), n_frames)
    z = fbm(x, y) + 2.0
    return [(G.rot_z(yaw[f]), np.array([x[f], y[f], z[f]])) for f in range(n_frames)]


def rig_frames(fbm, n_frames, traj_seed, rig):
    veh = vehicle_poses(fbm, n_frames, traj_seed)
    entries = []
    for f, (Rv, tv) in enumerate(veh):
        for s, (_kind, off, yaw, pitch) in enumerate(rig):
            Rm = G.rot_z(np.deg2rad(yaw)) @ G.rot_y(np.deg2rad(-pitch))
            entries.append((s, f, pose_rows(Rv @ Rm, Rv @ np.asarray(off) + tv)))
    return make_frames(entries)


def cfg2(n_frames=64):
    scene, fbm = _cfg1_scene()
    params = S.material_params(np.random.default_rng((SEED_SCENE + 1, 1)), 32)
    sensors = [_rig_sensor(kind) for kind, *_ in RIG]
    frames = rig_frames(fbm, n_frames, SEED_TRAJ + 2, RIG)
    return Workload("cfg2_batched_8sensors_64frames", scene, sensors, frames, params, SEED_NOISE + 2)


def cfg3(n_frames=16):
    scene, fbm = _cfg1_scene()
    params = S.material_params(np.random.default_rng((SEED_SCENE + 3, 1)), 32)
    hidden = S.material_params(np.random.default_rng(SEED_HIDDEN), 32)
    sensors = [S.sensor_128ch(2048, r_min=0.5, r_max=200.0, d_max=200.0)]
    frames = rig_frames(fbm, n_frames, SEED_TRAJ + 2, [("spin128", (0.0, 0.0, 0.0), 0.0, 0.0)])
    return Workload("cfg3_diff_128ch_16frames", scene, sensors, frames, params, SEED_NOISE + 3,
                    hidden_params=hidden)


# ------------------------------------------------------------------- cfg 4

def city_scene(rng, half=2048.0, cell=2.0, n_buildings=20000, n_materials=64, keepout=None,
               keepout_r=20.0, amplitude=5.0):
    """Heightfield terrain plus extruded convex-polygon buildings.

    Footprints: 5-12 points at sorted random angles on an ellipse (convex by
    construction), one building per cell of a 28 m grid so that they cannot
    overlap; walls split into 4 m storeys, flat fan-triangulated roof."""
    fbm = G.ValueNoiseFBM(rng, half, amplitude=amplitude)
    mb = G.MeshBuilder()
    n_cells = int(round(2 * half / cell))
    tv, tt, (ix, iy) = G.grid_terrain(n_cells, half, fbm)
    patch = rng.integers(0, 4, size=(n_cells // 32 + 1, n_cells // 32 + 1))
    tmat = np.repeat(patch[iy // 32, ix // 32], 2).astype(np.uint16)
    mb.add(tv, tt, tmat, 0)
    del tv, tt
    gcell = 28.0
    ng = int(2 * half // gcell) - 1
    cand = rng.permutation(ng * ng)
    k = 0
    for idx in cand:
        if k >= n_buildings:
            break
        gy, gx = divmod(int(idx), ng)
        cx = -half + gcell * (gx + 1)
        cy = -half + gcell * (gy + 1)
        r = rng.uniform(5.0, 13.0)
        jitter = (gcell / 2 - 0.5 - r)
        c = np.array([cx, cy]) + rng.uniform(-1, 1, size=2) * max(jitter, 0.0)
        if keepout is not None and np.min(np.hypot(keepout[:, 0] - c[0], keepout[:, 1] - c[1])) < keepout_r + r:
            continue
        n = int(rng.integers(5, 13))
        ang = np.sort(rng.uniform(0, 2 * np.pi, size=n))
        ell = rng.uniform(0.6, 1.0)
        yaw = rng.uniform(0, 2 * np.pi)
        pts = np.stack([r * np.cos(ang), r * ell * np.sin(ang)], 1) @ G.rot_z(yaw)[:2, :2].T + c
        height = rng.uniform(8.0, 40.0)
        base = float(fbm(c[0], c[1])) - 1.0
        n_st = max(1, int(np.ceil(height / 4.0)))
        zs = base + np.linspace(0.0, height + 1.0, n_st + 1)
        verts = []
        for z in zs:
            for p in pts:
                verts.append([p[0], p[1], z])
        tris = []
        for s in range(n_st):
            for e in range(n):
                a0 = s * n + e
                a1 = s * n + (e + 1) % n
                b0 = a0 + n
                b1 = a1 + n
                tris.append([a0, a1, b1])
                tris.append([a0, b1, b0])
        top = n_st * n
        for e in range(1, n - 1):
            tris.append([top, top + e, top + e + 1])
        m = int(rng.integers(4, n_materials))
        mb.add(np.array(verts), np.array(tris), m, 1 + k)
        k += 1
    return Scene(*mb.build()), fbm


_CITY_CACHE = {}


def cfg4(n_frames=32, n_az=4096):
    if "scene" not in _CITY_CACHE:
        tx, ty, _ = trajectory(np.random.default_rng(SEED_TRAJ + 4), n_frames)
        keep = np.stack([tx, ty], 1)
        _CITY_CACHE["scene"] = city_scene(np.random.default_rng(SEED_SCENE + 4), keepout=keep)
    scene, fbm = _CITY_CACHE["scene"]
    params = S.material_params(np.random.default_rng((SEED_SCENE + 4, 1)), 64)
    hidden = S.material_params(np.random.default_rng(SEED_HIDDEN + 1), 64)
    sensors = [S.sensor_128ch(n_az, r_min=0.5, r_max=200.0, d_max=200.0,
                              divergence_rad=1e-4, n_subrays=7)]
    frames = rig_frames(fbm, n_frames, SEED_TRAJ + 4, [("spin128", (0.0, 0.0, 0.0), 0.0, 0.0)])
    return Workload("cfg4_city10M_128ch_7subrays", scene, sensors, frames, params, SEED_NOISE + 4,
                    hidden_params=hidden)


# ------------------------------------------------------------ small variants

def small_terrain(seed=77, n_cells=32, half=16.0, n_objects=12, n_frames=2, n_az=256,
                  n_subrays=1, divergence=0.0, range_exp=0.0):
    """A cfg1-shaped workload small enough for the oracle to cover every beam."""
    tx, ty, _ = trajectory(np.random.default_rng(seed + 1), n_frames, amp_max=6.0)
    keep = np.concatenate([np.stack([tx, ty], 1), [[0.0, 0.0]]], 0)
    scene, fbm = terrain_objects_scene(np.random.default_rng(seed), n_cells=n_cells, half=half,
                                       n_objects=n_objects, obj_half=half - 2.0, n_materials=8,
                                       keepout=keep, keepout_r=3.0, amplitude=1.0)
    params = S.material_params(np.random.default_rng((seed, 1)), 8)
    sensor = S.sensor_32ch(n_az, r_min=0.5, r_max=40.0, d_max=40.0, n_subrays=n_subrays,
                           divergence_rad=divergence, range_exp=range_exp)
    x, y, yaw = trajectory(np.random.default_rng(seed + 1), n_frames, amp_max=6.0)
    entries = []
    for f in range(n_frames):
        entries.append((0, f, pose_rows(G.rot_z(yaw[f]), [x[f], y[f], float(fbm(x[f], y[f])) + 1.5])))
    hidden = S.material_params(np.random.default_rng((seed, 2)), 8)
    return Workload(f"small_terrain_{n_cells}", scene, [sensor], make_frames(entries), params,
                    seed + 5, hidden_params=hidden)


def by_index(i: int) -> Workload:
    return [cfg0, cfg1, cfg2, cfg3, cfg4][i]()


def adjoint_tape(n: int, n_materials: int, seed: int, period: int = 1 << 15, octaves: float = 20.0):
    """A seeded adjoint tape drawn directly (no cast): per beam a forward valid
    flag (80 % set), a material in [0, n_materials + 3) (ids past the table
    select its last row), an incidence angle uniform on [0, 90] degrees (every
    97th an integer, every 1013th exactly 90), a range factor in [0.5, 2], a
    target intensity and a target valid flag (90 % set).  The targets grow
    along a sawtooth: within each `period` beams their scale rises by 2^octaves,
    so a running maximum keeps growing inside any run of consecutive beams."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 90.0, n).astype(np.float32)
    theta[::97] = np.floor(theta[::97])
    theta[::1013] = 90.0
    ramp = np.exp2(octaves * (np.arange(n) % period) / period)
    return {"valid": (rng.uniform(size=n) < 0.8).astype(np.uint8),
            "mat": rng.integers(0, n_materials + 3, n).astype(np.uint16),
            "theta_deg": theta,
            "rf": rng.uniform(0.5, 2.0, n).astype(np.float32),
            "target_I": (rng.uniform(0.0, 1.0, n) * ramp).astype(np.float32),
            "target_valid": (rng.uniform(size=n) < 0.9).astype(np.uint8),
            "params": S.material_params(rng, n_materials)}
