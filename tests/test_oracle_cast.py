"""Pins of the oracle's per-beam model: closed forms on planes (Sec. II-A range,
Sec. II-C incidence angle and Eq. 4, Sec. II-D Eq. 5), an exact-rational
brute-force second pass, invariants, and the exemption flags."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from scenes_tiny import (const_table, ground_quad, identity_frame, quads_scene, random_tris_scene, sensor,
                         wall_x)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _plane_run(oracle_lib, h, el_deg, az_deg, table, **kw):
    scene = quads_scene([ground_quad()])
    az = np.radians(np.asarray(az_deg, np.float64))
    el = -np.radians(np.asarray(el_deg, np.float64))
    s = sensor(az, el, r_min=0.1, r_max=5000.0, d_max=5000.0, RL_max=1e-6, **kw)
    return oracle_lib.cast(scene, [s], identity_frame((0.0, 0.0, h)), table, seed=1), s


def test_plane_range_and_angle_closed_form(oracle_lib):
    """Sensor at height h over z = 0, beam at depression phi: d = h / sin(phi)
    and theta = 90 deg - phi."""
    phis = np.array([0.5, 2.0, 5.0, 10.0, 30.0, 45.0, 60.0, 85.0, 89.5])
    azs = np.linspace(0, 350, phis.size)
    table = np.tile(np.arange(91, dtype=np.float64), (1, 1))  # T[k] = k -> I = theta in degrees
    r, _ = _plane_run(oracle_lib, 1.8, phis, azs, table)
    assert np.all(r.tri != oracle_lib.NO_HIT)
    want_d = 1.8 / np.sin(np.radians(phis))
    assert np.allclose(r.range, want_d, rtol=1e-6, atol=0)
    assert np.allclose(r.theta_deg, 90.0 - phis, atol=1e-5)
    assert np.allclose(r.intensity, 90.0 - phis, atol=1e-5)
    # the normal faces the sensor (sensor frame = world frame here)
    assert np.allclose(r.normal, [[0, 0, 1]] * phis.size, atol=1e-12)
    assert np.allclose(r.xyz[:, 2], -1.8, rtol=1e-6)


def test_plane_integer_degree_and_lambertian(oracle_lib):
    """At integer-degree incidence the lerp returns the table entry; with a pure
    Lambertian table (Eq. 4) I = g a cos(theta) up to the 1-degree lerp error."""
    phis = np.array([10.0, 20.0, 30.0, 45.0, 60.0, 75.0, 80.0])
    params = np.array([[0.6, 0.0, 5.0]], np.float32)
    T = oracle_lib.build_tables(params)
    r, _ = _plane_run(oracle_lib, 3.0, phis, np.zeros(phis.size), T, gain=2.0)
    k = np.round(90.0 - phis).astype(int)
    assert np.allclose(r.R, T[0, k], atol=1e-7)
    assert np.allclose(r.intensity, 2.0 * T[0, k], atol=2e-7)
    a = float(np.float32(0.6))
    # general angles: |lerp - a cos| <= a * (1 deg)^2 / 8
    phis2 = np.linspace(1.3, 88.7, 40)
    r2, _ = _plane_run(oracle_lib, 3.0, phis2, np.zeros(phis2.size), T)
    th = np.radians(90.0 - phis2)
    assert np.all(np.abs(r2.intensity - a * np.cos(th)) <= a * np.radians(1.0) ** 2 / 8 + 1e-9)


def test_constant_table_gives_gain_times_constant(oracle_lib):
    phis = np.linspace(2, 88, 30)
    r, _ = _plane_run(oracle_lib, 2.0, phis, np.linspace(0, 300, 30), const_table(0.37), gain=1.5)
    assert np.allclose(r.intensity, 1.5 * 0.37, rtol=1e-15)


def test_inverse_square_with_range_exponent(oracle_lib):
    """p = 2: at fixed incidence angle, I * d^2 is constant (= g R r_ref^2)."""
    T = const_table(0.5)
    vals = []
    for h in (1.0, 2.0, 4.0, 8.0):
        r, _ = _plane_run(oracle_lib, h, [30.0], [0.0], T, range_exp=2.0, r_ref=1.0)
        vals.append(r.intensity[0] * r.range[0] ** 2)
    assert np.allclose(vals, 0.5, rtol=1e-12)


def _load_golden_capability():
    consts, rows = {}, []
    with open(os.path.join(GOLDEN, "capability_os0_128.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            a, b = line.split()
            if a in ("d_max", "RL_max"):
                consts[a] = float(b)
            else:
                rows.append((float(a), float(b)))
    return consts, rows


def test_capability_model_paper_constants(oracle_lib):
    """Eq. 5 with the paper's OS0-128 constants: detected iff R_L(d) <= R."""
    consts, rows = _load_golden_capability()
    for d, RL in rows:
        scene = quads_scene([wall_x(d)])
        s = sensor([0.0], [0.0], r_min=0.5, r_max=100.0, d_max=consts["d_max"], RL_max=consts["RL_max"])
        fr = identity_frame()
        above = oracle_lib.cast(scene, [s], fr, const_table(RL * (1 + 1e-4)), seed=0)
        below = oracle_lib.cast(scene, [s], fr, const_table(RL * (1 - 1e-4)), seed=0)
        assert above.range[0] == pytest.approx(d, rel=1e-12)
        assert above.valid[0] == 1, d
        assert below.valid[0] == 0, d
        assert below.tri[0] != oracle_lib.NO_HIT
    # the comparison is inclusive: R exactly at the threshold is detected
    scene = quads_scene([wall_x(25.0)])
    s = sensor([0.0], [0.0], r_min=0.5, r_max=100.0, d_max=50.0, RL_max=0.8)
    r0 = oracle_lib.cast(scene, [s], identity_frame(), const_table(0.5), seed=0)
    thr = float(np.float32(0.8)) * r0.range[0] / 50.0
    assert oracle_lib.cast(scene, [s], identity_frame(), const_table(thr), seed=0).valid[0] == 1
    assert oracle_lib.cast(scene, [s], identity_frame(), const_table(np.nextafter(thr, 0)), seed=0).valid[0] == 0
    # beyond d_max: dropped even for a perfect reflector (the search range ends
    # at min(r_max, d_max) + 9 sigma, so with sigma = 0.1 the wall is still hit)
    scene = quads_scene([wall_x(50.5)])
    s = sensor([0.0], [0.0], r_min=0.5, r_max=100.0, d_max=50.0, RL_max=0.8, sigma=0.1)
    r = oracle_lib.cast(scene, [s], identity_frame(), const_table(1.0), seed=0)
    assert r.valid[0] == 0 and r.tri[0] != oracle_lib.NO_HIT
    s = sensor([0.0], [0.0], r_min=0.5, r_max=100.0, d_max=50.0, RL_max=0.8, sigma=0.0)
    r = oracle_lib.cast(scene, [s], identity_frame(), const_table(1.0), seed=0)
    assert r.valid[0] == 0 and r.tri[0] == oracle_lib.NO_HIT


def test_min_range_drops_but_occludes(oracle_lib):
    scene = quads_scene([wall_x(0.3), wall_x(5.0)])
    s = sensor([0.0], [0.01], r_min=0.5, r_max=100.0, d_max=100.0, RL_max=0.8)
    r = oracle_lib.cast(scene, [s], identity_frame(), const_table(1.0), seed=0)
    assert r.valid[0] == 0
    assert r.tri[0] in (0, 1)          # the near wall, not the far one
    assert r.range[0] == pytest.approx(0.3 / math.cos(0.01), rel=1e-6)


def test_miss_and_noise(oracle_lib):
    scene = quads_scene([ground_quad(half=10.0)])
    s = sensor([0.0, 0.0], [-0.3, 0.3], r_min=0.1, r_max=100.0, d_max=100.0, RL_max=0.01, sigma=0.05)
    r = oracle_lib.cast(scene, [s], identity_frame((0, 0, 2.0)), const_table(0.9), seed=11)
    assert r.tri[1] == oracle_lib.NO_HIT and r.valid[1] == 0 and np.isinf(r.t[1])
    # d = t + sigma z with z the beam's Philox/Box-Muller draw
    z = oracle_lib.normal(11, 0, 0, 0, 0)
    assert r.range[0] == pytest.approx(r.t[0] + float(np.float32(0.05)) * z, rel=1e-14)


def _exact_hit(o, d, v0, v1, v2):
    """Exact rational ray/closed-triangle intersection by Cramer's rule on
    o + t d = v0 + u (v1 - v0) + v (v2 - v0).  Returns t or None."""
    e1 = [v1[i] - v0[i] for i in range(3)]
    e2 = [v2[i] - v0[i] for i in range(3)]
    b = [o[i] - v0[i] for i in range(3)]
    cols = [e1, e2, [-x for x in d]]

    def det3(c0, c1, c2):
        return (c0[0] * (c1[1] * c2[2] - c1[2] * c2[1]) - c1[0] * (c0[1] * c2[2] - c0[2] * c2[1])
                + c2[0] * (c0[1] * c1[2] - c0[2] * c1[1]))

    D = det3(*cols)
    if D == 0:
        return None
    u = det3(b, cols[1], cols[2]) / D
    v = det3(cols[0], b, cols[2]) / D
    t = det3(cols[0], cols[1], b) / D
    if u >= 0 and v >= 0 and u + v <= 1:
        return t
    return None


def test_exact_rational_second_pass(oracle_lib):
    rng = np.random.default_rng(9)
    scene = random_tris_scene(rng, n=25)
    az, el = synth.spinning_pattern(np.linspace(-40, 30, 10), 36)
    s = sensor(az, el, r_min=0.0, r_max=50.0, d_max=50.0, RL_max=1e-9)
    r = oracle_lib.cast(scene, [s], identity_frame(), const_table(0.5), seed=0)
    dirs = oracle_lib.beam_dirs(az, el)
    V = [[Fraction(float(x)) for x in v] for v in scene.verts]
    o = [Fraction(0)] * 3
    T_max = Fraction(float(np.float32(50.0)))  # sigma = 0
    n_flag = 0
    n_hit = 0
    for b in range(az.size):
        d = [Fraction(float(x)) for x in dirs[b]]
        best = None
        for k, (i0, i1, i2) in enumerate(scene.tris):
            t = _exact_hit(o, d, V[i0], V[i1], V[i2])
            if t is None or not (t > Fraction(1, 10000) and t <= T_max):
                continue
            if best is None or t < best[0]:
                best = (t, k)
        if r.flags[b] & (oracle_lib.FLAG_EDGE | oracle_lib.FLAG_TIE):
            n_flag += 1
            continue
        if best is None:
            assert r.tri[b] == oracle_lib.NO_HIT
        else:
            n_hit += 1
            assert r.tri[b] == best[1], b
            assert r.t[b] == pytest.approx(float(best[0]), rel=1e-12)
    assert n_hit > 100
    assert n_flag <= 0.02 * az.size


def test_edge_and_tie_flags(oracle_lib):
    # a beam straight down the shared diagonal of the ground quad's two triangles
    scene = quads_scene([ground_quad(half=10.0)])
    s = sensor([math.radians(45.0), math.radians(10.0)], [-math.radians(30.0)] * 2, r_min=0.1, r_max=100.0,
               d_max=100.0, RL_max=1e-6)
    r = oracle_lib.cast(scene, [s], identity_frame((0.0, 0.0, 2.0)), const_table(0.5), seed=0)
    assert r.flags[0] & oracle_lib.FLAG_EDGE
    assert not (r.flags[1] & oracle_lib.FLAG_EDGE)
    # two coincident copies of a wall: equal depth, lowest index wins, flagged as a tie
    scene = quads_scene([wall_x(7.0), wall_x(7.0)])
    s = sensor([0.05], [0.05], r_min=0.1, r_max=100.0, d_max=100.0, RL_max=1e-6)
    r = oracle_lib.cast(scene, [s], identity_frame(), const_table(0.5), seed=0)
    assert r.flags[0] & oracle_lib.FLAG_TIE
    assert r.tri[0] in (0, 1)


def _small_workload(**kw):
    return synth.small_terrain(n_cells=24, half=12.0, n_objects=8, n_frames=1, n_az=96, **kw)


def _flag_free(*rs):
    m = np.ones(rs[0].valid.size, bool)
    for r in rs:
        m &= (r.flags & 7) == 0
    return m


def test_rigid_motion_invariance(oracle_lib):
    """A rigid motion applied to scene and pose leaves range, angle, intensity,
    labels and the sensor-frame normal unchanged.  The motion is chosen so that
    the transformed FP32 inputs are exact (a cyclic axis permutation plus an
    integer shift of a scene quantised to 2^-12 m), so any difference is the
    oracle's own rounding."""
    w = _small_workload()
    T = oracle_lib.build_tables(w.params)
    q = 4096.0
    verts = (np.round(w.scene.verts.astype(np.float64) * q) / q).astype(np.float32)
    base = synth.Scene(verts, w.scene.tris, w.scene.mat, w.scene.inst)
    fr0 = w.frames.copy()
    for k in range(len(fr0)):
        P = fr0[k]["pose"].astype(np.float64).reshape(3, 4)
        P[:, 3] = np.round(P[:, 3] * q) / q
        fr0[k]["pose"] = P.reshape(12).astype(np.float32)
    r0 = oracle_lib.cast(base, w.sensors, fr0, T, w.seed)
    Q = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    s = np.array([37.0, -21.0, 5.0])
    moved = synth.Scene((verts.astype(np.float64) @ Q.T + s).astype(np.float32), w.scene.tris, w.scene.mat,
                        w.scene.inst)
    assert np.array_equal((moved.verts.astype(np.float64) - s) @ Q, verts.astype(np.float64))
    fr1 = fr0.copy()
    for k in range(len(fr1)):
        P = fr0[k]["pose"].astype(np.float64).reshape(3, 4)
        fr1[k]["pose"] = synth.pose_rows(Q @ P[:, :3], Q @ P[:, 3] + s)
    r1 = oracle_lib.cast(moved, w.sensors, fr1, T, w.seed)
    m = _flag_free(r0, r1)
    assert m.mean() > 0.97
    assert np.array_equal(r0.tri[m], r1.tri[m])
    assert np.array_equal(r0.inst[m], r1.inst[m])
    assert np.array_equal(r0.valid[m], r1.valid[m])
    h = m & (r0.tri != oracle_lib.NO_HIT)
    assert h.sum() > 1000
    assert np.allclose(r0.t[h], r1.t[h], rtol=1e-12)
    assert np.allclose(r0.theta_deg[h], r1.theta_deg[h], atol=1e-9)
    assert np.allclose(r0.intensity[h], r1.intensity[h], rtol=1e-10, atol=1e-13)
    assert np.allclose(r0.normal[h], r1.normal[h], atol=1e-12)
    assert np.allclose(r0.xyz[h], r1.xyz[h], rtol=1e-12, atol=1e-12)


def test_triangle_permutation_invariance(oracle_lib):
    w = _small_workload()
    T = oracle_lib.build_tables(w.params)
    r0 = oracle_lib.cast(w.scene, w.sensors, w.frames, T, w.seed)
    perm = np.random.default_rng(3).permutation(w.scene.n_tris)
    sc = synth.Scene(w.scene.verts, w.scene.tris[perm], w.scene.mat[perm], w.scene.inst[perm])
    r1 = oracle_lib.cast(sc, w.sensors, w.frames, T, w.seed)
    m = _flag_free(r0, r1)
    h1 = r1.tri != oracle_lib.NO_HIT
    mapped = np.where(h1, perm[np.minimum(r1.tri, perm.size - 1)], oracle_lib.NO_HIT)
    assert np.array_equal(r0.tri[m], mapped[m])
    assert np.array_equal(r0.t[m], r1.t[m])
    assert np.array_equal(r0.intensity[m], r1.intensity[m])


def test_subray_strongest_return(oracle_lib):
    w = synth.small_terrain(n_cells=24, half=12.0, n_objects=8, n_frames=1, n_az=64, n_subrays=7,
                            divergence=2e-2)
    T = oracle_lib.build_tables(w.params)
    r = oracle_lib.cast(w.scene, w.sensors, w.frames, T, w.seed)
    assert r.sub_I.shape[1] == 7
    anyv = r.sub_valid.any(1)
    assert np.array_equal(r.valid.astype(bool), anyv)
    I = np.where(r.sub_valid == 1, r.sub_I, -1.0)
    k = I.argmax(1)  # first maximum = lowest sub-ray index on ties
    assert np.array_equal(r.sub[anyv], k[anyv])
    assert np.array_equal(r.intensity[anyv], I[anyv, k[anyv]])
    assert np.all(r.sub[~anyv] == 0)
    # sub-ray 0 is the beam itself: same result as a single-ray sensor
    w1 = synth.small_terrain(n_cells=24, half=12.0, n_objects=8, n_frames=1, n_az=64)
    r1 = oracle_lib.cast(w1.scene, w1.sensors, w1.frames, T, w1.seed)
    assert np.array_equal(r1.tri, r.sub_tri[:, 0])
    assert np.array_equal(r1.intensity, r.sub_I[:, 0])


def test_cfg0_flag_rates(oracle_lib):
    w = synth.cfg0()
    T = oracle_lib.build_tables(w.params)
    r = oracle_lib.cast(w.scene, w.sensors, w.frames, T, w.seed)
    assert r.valid.sum() > 5000
    assert ((r.flags & 7) != 0).mean() < 0.01


def test_range_scaled_noise_closed_form(oracle_lib):
    """Range-scaled noise (the noise factor of Sec. II-A growing with range):
    d = t + (sigma + sigma_k t) z, with z the Box-Muller draw of the beam's
    Philox4x64-10 block (counter (beam, frame | sensor << 32, sub-ray, 0), key
    (seed, 0)) computed here from numpy's Philox."""
    from test_oracle_pieces import _numpy_philox_block
    h, seed = 1.8, 77
    phis = np.array([1.0, 3.0, 8.0, 20.0, 45.0, 80.0])
    sig, sk = 0.02, 0.004
    scene = quads_scene([ground_quad()])
    s = sensor(np.linspace(0, 6, phis.size), -np.radians(phis), r_min=0.01, r_max=500.0, d_max=500.0,
               RL_max=1e-6, sigma=sig, sigma_k=sk)
    r = oracle_lib.cast(scene, [s], identity_frame((0.0, 0.0, h), frame=5), const_table(0.5), seed=seed)
    t = r.t
    assert np.allclose(t, h / np.sin(np.radians(phis)), rtol=1e-6)
    z = []
    for b in range(phis.size):
        x = _numpy_philox_block([b, 5 | (0 << 32), 0, 0], [seed, 0])
        u0 = ((int(x[0]) >> 11) + 0.5) * 2.0 ** -53
        u1 = ((int(x[1]) >> 11) + 0.5) * 2.0 ** -53
        z.append(math.sqrt(-2.0 * math.log(u0)) * math.cos(2.0 * math.pi * u1))
    z = np.array(z)
    s32, k32 = float(np.float32(sig)), float(np.float32(sk))
    assert np.allclose(r.range, t + (s32 + k32 * t) * z, rtol=1e-12, atol=1e-12)


def test_range_scaled_noise_search_range(oracle_lib):
    """With sigma_k > 0 the search range is (d_lim + 9 sigma) / (1 - 9 sigma_k):
    a wall just inside it is hit, one just beyond it is a miss."""
    sig, sk, dlim = 0.05, 0.02, 100.0
    T = (float(np.float32(dlim)) + 9.0 * float(np.float32(sig))) / (1.0 - 9.0 * float(np.float32(sk)))
    for x, hit in ((T * (1 - 1e-4), True), (T * (1 + 1e-4), False)):
        scene = quads_scene([wall_x(x, half=10.0)])
        s = sensor(np.zeros(1), np.zeros(1), r_min=0.5, r_max=dlim, d_max=dlim, RL_max=1e-6, sigma=sig, sigma_k=sk)
        r = oracle_lib.cast(scene, [s], identity_frame(), const_table(0.5), seed=1)
        assert (r.tri[0] != oracle_lib.NO_HIT) == hit


def _with_degenerates(scene, tris_xyz):
    """`scene` plus triangles given by their three vertices (appended after it,
    so the original triangles keep their indices)."""
    v0 = scene.verts.shape[0]
    verts = np.concatenate([scene.verts, np.asarray(tris_xyz, np.float32).reshape(-1, 3)])
    k = len(tris_xyz)
    tris = np.concatenate([scene.tris, (v0 + np.arange(3 * k, dtype=np.uint32)).reshape(k, 3)])
    mat = np.concatenate([scene.mat, np.zeros(k, np.uint16)])
    inst = np.concatenate([scene.inst, np.full(k, 99, np.uint32)])
    return synth.Scene(verts, tris, mat, inst)


def test_degenerate_triangles_are_never_hit(oracle_lib):
    """Zero-area triangles — one point three times, or two equal vertices and a
    third — placed exactly on the beams' paths are never hit: the beams reach
    the wall x = 20 behind them (range 20 / cos of the azimuth in the plane)."""
    wall = quads_scene([wall_x(20.0, half=200.0)])
    az = np.radians([0.0, 0.0, 10.0, -7.5])
    el = np.zeros(4)
    s = sensor(az, el, r_min=0.1, r_max=500.0, d_max=500.0, RL_max=1e-6)
    d = oracle_lib.beam_dirs(s.az_rad, s.el_rad).astype(np.float64)
    pts = [np.float32(10.0) * d[i].astype(np.float32) for i in range(4)]      # points on (or next to) the beams
    degs = [[p, p, p] for p in pts] + [[p, p, p + np.float32([0.0, 0.0, 3.0])] for p in pts] + \
        [[(10.0, -5.0, 0.0), (10.0, 5.0, 0.0), (10.0, -5.0, 0.0)]]             # a repeated-vertex segment across beam 0
    scene = _with_degenerates(wall, degs)
    r = oracle_lib.cast(scene, [s], identity_frame(), const_table(0.5), 1)
    assert np.all(r.tri < 2)                                                  # a wall triangle, never a degenerate one
    assert np.allclose(r.range, 20.0 / d[:, 0], rtol=1e-12)
    base = oracle_lib.cast(wall, [s], identity_frame(), const_table(0.5), 1)
    assert np.array_equal(r.tri, base.tri) and np.array_equal(r.range, base.range)
