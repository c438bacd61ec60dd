"""Pins of the oracle's raster-and-resample path (the paper's own sampling,
Sec. II-A..II-C): camera intrinsics of Eq. 1-2, the corrected pixel equations
of Eq. 3, the depth pass as z-depth in three bytes, the incidence angle, the
8-bit material stencil and the 24-bit instance colour, and the depth read back
along the beam — each against a closed form on planes."""
import math

import numpy as np

import synth
from scenes_tiny import const_table, ground_quad, identity_frame, quads_scene, sensor, wall_x

Q24 = 16777215.0


def test_camera_constants_closed_form(oracle_lib):
    for W, K in ((1024, 6), (512, 4), (640, 5)):
        f, c, ck, sk = oracle_lib.raster_constants(W, K)
        assert f == float(np.float32(W / (2.0 * math.tan(math.pi / K))))   # Eq. 2, FOV_c = 360/K degrees
        assert c == W / 2.0
        az = -math.pi + (np.arange(K) + 0.5) * 2.0 * math.pi / K
        assert np.array_equal(ck, np.cos(az).astype(np.float32))
        assert np.array_equal(sk, np.sin(az).astype(np.float32))


def _wall_run(oracle_lib, D, az_deg, el_deg, W=640, K=5):
    # K = 5 puts camera 2 on the +x axis; the wall x = D is perpendicular to it
    scene = quads_scene([wall_x(D, half=400.0)])
    s = sensor(np.radians(az_deg), np.radians(el_deg), r_min=0.1, r_max=300.0, d_max=300.0, RL_max=1e-6)
    fr = identity_frame((0.0, 0.0, 0.0))
    T = const_table(0.5)
    return (oracle_lib.raster(scene, [s], fr, T, 3, W, K), oracle_lib.cast(scene, [s], fr, T, 3), s)


def test_fronto_parallel_wall_depth_and_range(oracle_lib):
    """A wall perpendicular to the camera axis has the same z-depth D at every
    pixel, so the pixel read along the beam gives the beam's exact range up to
    the 24-bit depth step: range = q T_max / (2^24 - 1) / (d . F)."""
    D = 37.25
    az = np.array([-30.0, -17.3, -5.0, 0.0, 0.7, 12.0, 29.0])
    el = np.array([-20.0, -8.0, 3.0, 0.0, 10.5, -1.0, 15.0])
    r, c, s = _wall_run(oracle_lib, D, az, el)
    T_max = float(np.float32(np.float32(300.0) + np.float32(9.0) * np.float32(0.0)))
    assert np.all(r.cam == 2) and not r.outside.any()
    assert np.allclose(r.z, D, rtol=1e-7)
    q = np.rint(np.float32(D) * np.float32(np.float32(Q24) / np.float32(T_max))).astype(np.float64)
    assert np.all(r.q_depth == q)
    d = oracle_lib.beam_dirs(s.az_rad, s.el_rad)
    want = (q * T_max / Q24) / d[:, 0].astype(np.float64)       # F = +x
    assert np.allclose(r.range, want, rtol=1e-12)
    # and that is the ray-cast range to within one depth step along the beam
    assert np.all(np.abs(r.range - c.range) <= (T_max / Q24) / d[:, 0] + 1e-9 * c.range)


def test_wall_incidence_angle_from_pixel_centre(oracle_lib):
    """On the wall the angle between the pixel-centre ray and the normal is
    atan(sqrt(a^2 + b^2)) with (a, b) the pixel centre's offsets over f."""
    az = np.array([-25.0, -3.0, 0.0, 8.0, 21.0])
    el = np.array([5.0, -12.0, 0.0, 2.0, -7.0])
    r, _, _ = _wall_run(oracle_lib, 20.0, az, el)
    f, c, _, _ = oracle_lib.raster_constants(640, 5)
    a = (r.px + 0.5 - c) / f
    b = (c - (r.py + 0.5)) / f
    theta = np.degrees(np.arctan(np.hypot(a, b)))
    assert np.all(np.abs(r.theta_deg - theta) <= 90.0 / Q24 + 1e-6)
    assert np.all(np.abs(r.q_angle - np.rint(theta * Q24 / 90.0)) <= 1)


def test_pixel_indices_closed_form(oracle_lib):
    """n_x = c + f tan(delta), n_y = c - f tan(phi) / cos(delta) (corrected
    Eq. 3; image rows grow downwards), pixel = floor."""
    az = np.array([-31.0, -10.0, 0.3, 7.7, 33.0])
    el = np.array([-25.0, -2.2, 0.05, 9.0, 20.0])
    r, _, _ = _wall_run(oracle_lib, 50.0, az, el)
    f, c, _, _ = oracle_lib.raster_constants(640, 5)
    dl, ph = np.radians(az), np.radians(el)
    nx = c + f * np.tan(dl)
    ny = c - f * np.tan(ph) / np.cos(dl)
    assert np.array_equal(r.px, np.floor(nx).astype(np.int32))
    assert np.array_equal(r.py, np.floor(ny).astype(np.int32))


def test_ground_plane_row_depth(oracle_lib):
    """Sensor at height h over z = 0: the pixel-centre ray of row j has
    y/z = b = (c - (j + 1/2)) / f, so its z-depth is h / (-b) exactly; the beam
    then reads that depth along its own direction."""
    h = 2.0
    phis = np.array([2.0, 4.0, 7.5, 12.0, 20.0, 30.0])
    scene = quads_scene([ground_quad()])
    s = sensor(np.zeros(phis.size), -np.radians(phis), r_min=0.1, r_max=300.0, d_max=300.0, RL_max=1e-6)
    T = const_table(0.5)
    r = oracle_lib.raster(scene, [s], identity_frame((0.0, 0.0, h)), T, 3, 640, 5)
    f, c, _, _ = oracle_lib.raster_constants(640, 5)
    b = (np.float32(c) - (r.py.astype(np.float32) + np.float32(0.5))) / np.float32(f)
    assert np.all(r.px == 320)
    assert np.allclose(r.z, h / -b.astype(np.float64), rtol=1e-6)
    d = oracle_lib.beam_dirs(s.az_rad, s.el_rad)
    zq = r.q_depth * (float(np.float32(300.0)) / Q24)
    assert np.allclose(r.range, zq / d[:, 0], rtol=1e-12)
    # the sampling error: the beam's true range h / sin(phi) differs from the
    # pixel's depth read along it by at most one pixel row of depth
    true = h / np.sin(np.radians(phis))
    row_step = h / -b - h / -(b - 1.0 / f)
    assert np.all(np.abs(r.range - true) <= np.abs(row_step) / d[:, 0] + 1e-4)


def test_stencil_material_and_colour_instance(oracle_lib):
    """The material stencil keeps 8 bits and the instance colour 24 bits."""
    scene = quads_scene([wall_x(10.0)], materials=[300], instances=[0x1234567])
    M = 64
    table = np.tile(np.linspace(0.1, 0.9, 91), (M, 1)) * (np.arange(M)[:, None] + 1) / M
    s = sensor(np.radians([0.0, 5.0]), np.radians([0.0, -3.0]), r_min=0.1, r_max=300.0, d_max=300.0,
               RL_max=1e-6)
    r = oracle_lib.raster(scene, [s], identity_frame(), table, 3, 640, 5)
    assert np.all(r.mat == 300 & 0xFF)
    assert np.all(r.inst == 0x234567)
    row = table[44]
    i = np.minimum(np.floor(r.theta_deg).astype(int), 89)
    fr = r.theta_deg - i
    assert np.allclose(r.intensity, row[i] * (1 - fr) + row[i + 1] * fr, rtol=1e-12)


def test_beams_outside_the_camera_rows(oracle_lib):
    """A beam steeper than the camera's half field (36 degrees for K = 5) projects
    outside the image: no return."""
    r, _, _ = _wall_run(oracle_lib, 20.0, np.array([0.0, 0.0, 10.0]), np.array([40.0, -50.0, 30.0]))
    assert list(r.outside) == [1, 1, 0]
    assert not r.valid[:2].any() and np.all(r.tri[:2] == 0xFFFFFFFF)


def test_camera_border_beams_clamp_to_the_edge_column(oracle_lib):
    """Beams exactly between two cameras (azimuth 0 with K = 6) belong to the
    lower-indexed camera and read its last column."""
    scene = quads_scene([wall_x(15.0)])
    s = sensor(np.radians([0.0, 0.0]), np.radians([0.0, 4.0]), r_min=0.1, r_max=300.0, d_max=300.0,
               RL_max=1e-6)
    r = oracle_lib.raster(scene, [s], identity_frame(), const_table(0.5), 3, 512, 6)
    assert not r.outside.any()
    assert np.all(r.cam == 2) and np.all(r.px == 511)


def test_raster_agrees_with_ray_cast_on_cfg0(oracle_lib):
    """On the boxes scene the raster path sees the beam's own triangle for all
    but a thin silhouette band, and its range differs from the ray cast by the
    sub-pixel sampling error (median well below the noise sigma)."""
    w = synth.cfg0()
    T = oracle_lib.build_tables(w.params)
    r = oracle_lib.raster(w.scene, w.sensors, w.frames, T, w.seed, 512, 6)
    c = oracle_lib.cast(w.scene, w.sensors, w.frames, T, w.seed)
    assert not r.outside.any()
    both = (r.tri != 0xFFFFFFFF) & (c.tri != 0xFFFFFFFF)
    assert (r.tri[both] == c.tri[both]).mean() > 0.99
    assert np.median(np.abs(r.range[both] - c.range[both])) < 0.05
