"""Pins of the oracle's rolling shutter (the sensor turns over each time step,
Sec. II-A) and multi-echo returns (Sec. IV future work), against closed
forms: firing fractions, quaternions of known rotations, interpolated poses,
ranges seen by a moving sensor, and echo choices on a two-wall edge."""
import math

import numpy as np

import synth
from scenes_tiny import const_table, quads_scene, sensor, wall_x


def _rot(axis, ang):
    c, s = math.cos(ang), math.sin(ang)
    if axis == "x":
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    if axis == "y":
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def _pose(R, t=(0.0, 0.0, 0.0)):
    return synth.pose_rows(np.asarray(R, np.float64), t)


def test_sweep_fraction(oracle_lib):
    for az, s in ((0.0, 0.0), (math.pi, 0.5), (-math.pi / 2, 0.75), (2 * math.pi, 0.0), (5 * math.pi, 0.5)):
        assert oracle_lib.sweep_fraction(az) == float(np.float32(s))


def test_quaternions_of_known_rotations(oracle_lib):
    """Shepperd's four branches: identity, a 90-degree yaw, and half turns
    about x, y and z (unit quaternion (w, x, y, z), w >= 0 on those)."""
    h = math.sqrt(0.5)
    cases = [(np.eye(3), (1, 0, 0, 0)), (_rot("z", math.pi / 2), (h, 0, 0, h)), (_rot("x", math.pi), (0, 1, 0, 0)),
             (_rot("y", math.pi), (0, 0, 1, 0)), (_rot("z", math.pi), (0, 0, 0, 1))]
    for R, q in cases:
        q0, _ = oracle_lib.sweep_quaternions(_pose(R), _pose(np.eye(3)))
        assert np.allclose(np.abs(q0), np.abs(np.array(q, np.float32)), atol=1e-7), (R, q0)


def test_pose_reconstruction_and_interpolation(oracle_lib):
    rng = np.random.default_rng(3)
    for _ in range(20):
        # random rotation from a random unit quaternion
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        t0, t1 = rng.uniform(-50, 50, 3), rng.uniform(-50, 50, 3)
        p0, p1 = _pose(R, t0), _pose(R @ _rot("z", 0.3), t1)
        A = oracle_lib.sweep_pose(p0, p1, 0.0).reshape(3, 4)
        B = oracle_lib.sweep_pose(p0, p1, 1.0).reshape(3, 4)
        assert np.allclose(A[:, :3], p0.reshape(3, 4)[:, :3], atol=2e-6)
        assert np.allclose(B[:, :3], p1.reshape(3, 4)[:, :3], atol=2e-6)
        assert np.array_equal(A[:, 3], p0.reshape(3, 4)[:, 3])
        assert np.array_equal(B[:, 3], p1.reshape(3, 4)[:, 3])
    # the midpoint of a yaw from 0 to 90 degrees is the 45-degree yaw (normalised
    # blend and spherical interpolation agree there), translation halfway
    M = oracle_lib.sweep_pose(_pose(np.eye(3), (0, 0, 0)), _pose(_rot("z", math.pi / 2), (2, 4, 0)), 0.5)
    M = M.reshape(3, 4)
    assert np.allclose(M[:, :3], _rot("z", math.pi / 4), atol=1e-6)
    assert np.array_equal(M[:, 3], np.float32([1, 2, 0]))


def test_rolling_shutter_translating_sensor(oracle_lib):
    """The sensor moves from y = 0 to y = Delta during the sweep in front of the
    wall y = D: the beam at azimuth a fires at s = a / 2 pi, from y = s Delta,
    so its range is (D - s Delta) / sin(a)."""
    D, delta = 30.0, 4.0
    wall = [(-100.0, D, -50.0), (100.0, D, -50.0), (100.0, D, 50.0), (-100.0, D, 50.0)]
    az = np.radians([20.0, 45.0, 90.0, 120.0, 160.0])
    s = sensor(az, np.zeros(az.size), r_min=0.1, r_max=500.0, d_max=500.0, RL_max=1e-6)
    fr = synth.make_sweep_frames([(0, 0, _pose(np.eye(3), (0, 0, 0)), _pose(np.eye(3), (0, delta, 0)))])
    r = oracle_lib.cast_sweep(quads_scene([wall]), [s], fr, const_table(0.5), 1)
    frac = np.array([oracle_lib.sweep_fraction(a) for a in az])
    assert np.allclose(r.range, (D - frac * delta) / np.sin(az), rtol=1e-6)


def test_static_sweep_equals_frame_cast(oracle_lib):
    w = synth.cfg0()
    T = oracle_lib.build_tables(w.params)
    p = w.frames[0]["pose"]
    fr = synth.make_sweep_frames([(0, int(w.frames[0]["frame"]), p, p)])
    samples = (np.zeros(300, np.int64), np.arange(0, 28800, 96, dtype=np.int64))
    a = oracle_lib.cast_sweep(w.scene, w.sensors, fr, T, w.seed, samples=samples)
    b = oracle_lib.cast(w.scene, w.sensors, w.frames[:1], T, w.seed, samples=samples)
    assert np.array_equal(a.tri, b.tri) and np.array_equal(a.valid, b.valid)
    # the blended translation (1 - s) t0 + s t0 is t0 to within an ulp
    assert np.allclose(a.range, b.range, rtol=1e-6)


def _edge_scene():
    """Near wall x = 10 for y < 0 (material 0), far wall x = 20 for y >= 0
    (material 1); a table with R = 0.3 and 0.7 at every angle."""
    near = [(10.0, -50.0, -50.0), (10.0, 0.0, -50.0), (10.0, 0.0, 50.0), (10.0, -50.0, 50.0)]
    far = [(20.0, 0.0, -50.0), (20.0, 50.0, -50.0), (20.0, 50.0, 50.0), (20.0, 0.0, 50.0)]
    table = np.stack([np.full(91, 0.3), np.full(91, 0.7)])
    return quads_scene([near, far], materials=[0, 1]), table


def test_echoes_on_an_edge(oracle_lib):
    """A divergent beam aimed just beside the edge between a near dark wall and a
    far bright wall: sub-rays land on both.  Strongest first: the far wall
    (lowest sub-ray there), then the near wall; first/last: near then far; a
    separation larger than the walls' gap leaves one echo."""
    scene, table = _edge_scene()
    s = sensor(np.array([2e-4]), np.zeros(1), r_min=0.1, r_max=500.0, d_max=500.0, RL_max=1e-6,
               divergence_rad=2e-3, n_subrays=7)
    fr = synth.make_sweep_frames([(0, 0, _pose(np.eye(3)), _pose(np.eye(3)))])
    r0 = oracle_lib.cast_sweep(scene, [s], fr, table, 1, echoes=(2, 0, 1.0))
    far = np.flatnonzero(r0.sub_range[0] > 15.0)
    near = np.flatnonzero((r0.sub_range[0] < 15.0) & (r0.sub_valid[0] != 0))
    assert far.size and near.size
    assert r0.echo_count[0] == 2
    assert r0.echo_sub[0, 0] == far.min() and r0.echo_sub[0, 1] == near.min()
    assert np.isclose(r0.echo_intensity[0, 0], 0.7) and np.isclose(r0.echo_intensity[0, 1], 0.3)
    r1 = oracle_lib.cast_sweep(scene, [s], fr, table, 1, echoes=(2, 1, 1.0))
    rng = r1.sub_range[0]
    valid = r1.sub_valid[0] != 0
    assert r1.echo_count[0] == 2
    assert r1.echo_range[0, 0] == rng[valid].min() and r1.echo_range[0, 1] == rng[valid].max()
    r2 = oracle_lib.cast_sweep(scene, [s], fr, table, 1, echoes=(2, 1, 15.0))
    assert r2.echo_count[0] == 1 and r2.echo_range[0, 0] == rng[valid].min()


def test_echo_separation_merges_one_surface(oracle_lib):
    scene = quads_scene([wall_x(25.0)])
    s = sensor(np.array([0.3]), np.array([0.1]), r_min=0.1, r_max=500.0, d_max=500.0, RL_max=1e-6,
               divergence_rad=1e-3, n_subrays=7)
    fr = synth.make_sweep_frames([(0, 0, _pose(np.eye(3)), _pose(np.eye(3)))])
    r = oracle_lib.cast_sweep(scene, [s], fr, const_table(0.5), 1, echoes=(3, 0, 1.0))
    assert r.echo_count[0] == 1
