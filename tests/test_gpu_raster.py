"""GPU parity of the raster-and-resample path (the paper's own sampling,
Sec. II-A..II-C) against the oracle: every beam on small scenes, a seeded
sample of the full 128-channel frame, the G-buffer pixels themselves, and the
edge cases (empty scene, beams outside the camera rows, bad configurations).

Tolerances: triangle, material stencil, instance colour, valid mask and the
pixel a beam reads are bit-exact outside the counted exemptions (EDGE and TIE
of the pixel-centre ray, CUTOFF).  The 24-bit depth code is an integer
quantisation of a depth that the two sides compute differently (the GPU from
its FP32 watertight hit, the oracle from its FP64 hit rounded to FP32), so it
may differ by a bounded number of codes, derived per pixel: the FP32 hit's
position error is read at the scale of the EDGE band, 1e-6 max(|o|, |v|, t)
metres (o the pixel ray's origin, v the hit triangle's vertices, t the hit
distance); along the pixel ray the depth differs by at most that much, which
is dt q_s codes with q_s = (2^24 - 1) / T_max, plus one for the two roundings
to an integer.  Code differences are counted (0, 1, more) and reported.  The
range before noise, decoded from the code along the beam, may then differ by
that many depth steps plus the FP32 rounding of the decode (4 ulp).  The
angle code (three bytes over 90 degrees) within 1e-4 degrees, its differences
counted the same way; intensity 1e-4 relative.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import frame_offsets, setup, stratified_sample
from parity import to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REPORT = os.environ.get("LIDAR_PARITY_REPORT")
Q24 = 16777215.0
EXEMPT = 1 | 2 | 4


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_10295_gb300 import Lidar
    lid = Lidar(0)
    yield lid
    lid.close()


def _report(rep):
    print(json.dumps(rep))
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps(rep) + "\n")


FIELDS = ("valid", "tri", "t", "range", "intensity", "mat", "inst", "theta_deg")


def gpu_raster(L, w, width, n_cameras, scene=None):
    scene, _ = setup(L, w, scene)
    n = L.total_beams(w.frames)
    beams = L.alloc_beams(n, FIELDS)
    L.raster_cast_into(scene, w.frames, w.seed, beams, width=width, n_cameras=n_cameras)
    assert L.sync_status() == 0
    return to_numpy(beams), scene


def _t_max32(spec):
    """The search range in FP32 exactly as both sides form it (range-scaled noise included)."""
    f = np.float32
    return float((f(min(spec.r_max, spec.d_max)) + f(9.0) * f(spec.sigma)) /
                 (f(1.0) - f(9.0) * f(getattr(spec, "sigma_k", 0.0))))


def code_bound(w, frame_idx, tri, t_pix, T_max):
    """Largest depth-code difference the FP32 path may show at each pixel:
    ceil(1e-6 max(|o|inf, |v|inf, t) (2^24 - 1) / T_max) + 1."""
    o = np.abs(np.stack([np.asarray(w.frames[int(f)]["pose"], np.float64)[[3, 7, 11]] for f in frame_idx]))
    v = np.abs(w.scene.verts[w.scene.tris[tri]].astype(np.float64)).reshape(len(tri), -1)
    scale = np.maximum(np.maximum(o.max(1), v.max(1)), np.abs(t_pix))
    return np.ceil(1e-6 * scale * Q24 / T_max) + 1.0


def code_counts(d):
    d = np.abs(np.asarray(d, np.int64))
    return {"0": int((d == 0).sum()), "1": int((d == 1).sum()), ">1": int((d > 1).sum()),
            "max": int(d.max()) if d.size else 0}


def compare_raster(g, r, w, samples, label):
    """g: GPU dense fields at the samples; r: oracle.raster result."""
    flags = r.flags.astype(np.int64)
    ok = (flags & EXEMPT) == 0
    n = flags.size
    rep = {"label": label, "beams": int(n), "exempt": int((~ok).sum()), "outside": int(r.outside.sum())}
    bad = ok & (g["tri"] != r.tri)
    assert not bad.any(), f"{label}: pixel triangle differs on {int(bad.sum())} beams, e.g. {np.flatnonzero(bad)[:5]}"
    bad = ok & (g["valid"].astype(bool) != r.valid.astype(bool))
    assert not bad.any(), f"{label}: valid differs on {int(bad.sum())} beams, e.g. {np.flatnonzero(bad)[:5]}"
    h = ok & (r.tri != 0xFFFFFFFF)
    assert np.array_equal(g["mat"][h], r.mat[h]), f"{label}: stencil differs"
    assert np.array_equal(g["inst"][h], r.inst[h]), f"{label}: colour differs"
    T_max = np.array([_t_max32(w.sensors[int(w.frames[f]["sensor"])]) for f in samples[0]], np.float64)
    # range before noise: the oracle's is range - sigma z; recover it from its depth code
    sig = np.array([w.sensors[int(w.frames[f]["sensor"])].sigma for f in samples[0]], np.float64)
    zn = np.array([oracle.normal(w.seed, int(b), int(w.frames[f]["frame"]), int(w.frames[f]["sensor"]), 0)
                   for f, b in zip(*samples)]) if h.any() else np.zeros(n)
    t_or = r.range - sig * zn
    zq = r.q_depth[h] * T_max[h] / Q24              # decoded depth of the pixel
    step = (T_max[h] / Q24) * t_or[h] / zq           # one depth step along the beam
    kq = code_bound(w, samples[0][h], r.tri[h], r.t[h], T_max[h])
    dt = np.abs(g["t"][h].astype(np.float64) - t_or[h])
    rep["t_max_abs"] = float(dt.max()) if dt.size else 0.0
    rep["depth_codes_along_beam"] = code_counts(np.rint(dt / step))
    rep["code_bound_max"] = int(kq.max()) if kq.size else 0
    assert np.all(dt <= kq * step + 4 * 2.0 ** -24 * t_or[h]), \
        f"{label}: range before noise differs by {rep['t_max_abs']:.3g} (beyond the derived code bound)"
    dth = np.abs(g["theta_deg"][h].astype(np.float64) - r.theta_deg[h])
    rep["theta_max_abs"] = float(dth.max()) if dth.size else 0.0
    assert rep["theta_max_abs"] <= 1e-4, f"{label}: angle differs by {rep['theta_max_abs']:.3g}"
    dI = np.abs(g["intensity"][h].astype(np.float64) - r.intensity[h])
    rep["intensity_max_rel"] = float((dI / np.maximum(np.abs(r.intensity[h]), 1e-30)).max()) if dI.size else 0.0
    assert np.all(dI <= 1e-4 * np.abs(r.intensity[h]) + 1e-7), f"{label}: intensity differs"
    rep["hits"] = int(h.sum())
    rep["returns"] = int((h & (r.valid != 0)).sum())
    return rep


def _pick(g, w, samples):
    idx = frame_offsets(w)[samples[0]] + samples[1]
    return {k: v[idx] for k, v in g.items()}


@pytest.mark.parametrize("width,n_cameras", [(512, 6), (300, 5), (256, 3), (96, 64)])
def test_raster_cfg0_every_beam(L, width, n_cameras):
    w = synth.cfg0()
    g, _ = gpu_raster(L, w, width, n_cameras)
    T = oracle.build_tables(w.params)
    r = oracle.raster(w.scene, w.sensors, w.frames, T, w.seed, width, n_cameras)
    samples = (r.sample_frame, r.sample_beam)
    _report(compare_raster(_pick(g, w, samples), r, w, samples, f"raster cfg0 W={width} K={n_cameras}, every beam"))


def test_raster_small_terrain_every_beam(L):
    w = synth.small_terrain(seed=78, n_frames=2, n_az=256)
    g, _ = gpu_raster(L, w, 1024, 6)
    T = oracle.build_tables(w.params)
    r = oracle.raster(w.scene, w.sensors, w.frames, T, w.seed, 1024, 6)
    samples = (r.sample_frame, r.sample_beam)
    _report(compare_raster(_pick(g, w, samples), r, w, samples, "raster small terrain W=1024 K=6, every beam"))


def test_raster_cfg1_full_frame_sampled(L):
    w = synth.cfg1()
    g, _ = gpu_raster(L, w, 1024, 6)
    samples = stratified_sample(w, 4096, seed=5)
    T = oracle.build_tables(w.params)
    r = oracle.raster(w.scene, w.sensors, w.frames, T, w.seed, 1024, 6, samples=samples)
    _report(compare_raster(_pick(g, w, samples), r, w, samples, "raster cfg1 full frame W=1024 K=6, 4096 sampled"))
    # whole-frame properties: labels are the pixel triangle's labels (8/24-bit)
    hit = g["tri"] != 0xFFFFFFFF
    assert hit.sum() > 100000
    assert np.array_equal(g["inst"][hit], w.scene.inst[g["tri"][hit]] & 0xFFFFFF)
    assert np.array_equal(g["mat"][hit], w.scene.mat[g["tri"][hit]] & 0xFF)


def test_raster_gbuffer_pixels_match_oracle(L):
    """The G-buffer itself: at the pixels the oracle's beams read, the GPU's
    triangle, stencil and colour are the oracle's, the depth code within four
    steps and the angle code within 1e-4 degrees."""
    w = synth.small_terrain(seed=79, n_frames=1, n_az=256)
    scene, _ = setup(L, w)
    G = L.raster_gbuffer(scene, w.frames[:1], width=640, n_cameras=5)
    assert L.sync_status() == 0
    G = {k: v.cpu().numpy().view(np.uint32) for k, v in G.items()}
    T = oracle.build_tables(w.params)
    r = oracle.raster(w.scene, w.sensors, w.frames, T, w.seed, 640, 5)
    ok = ((r.flags & EXEMPT) == 0) & (r.outside == 0)
    k, y, x = r.cam[ok], r.py[ok], r.px[ok]
    assert np.array_equal(G["tri"][k, y, x], r.tri[ok])
    hit = r.tri[ok] != 0xFFFFFFFF
    kh, yh, xh = k[hit], y[hit], x[hit]
    # the depth codes, integers, compared directly against the derived per-pixel bound
    T_max = _t_max32(w.sensors[0])
    kq = code_bound(w, r.sample_frame[ok][hit], r.tri[ok][hit], r.t[ok][hit], T_max)
    dq = G["depth"][kh, yh, xh].astype(np.int64) - r.q_depth[ok][hit].astype(np.int64)
    assert np.all(np.abs(dq) <= kq), f"depth code beyond its bound: {code_counts(dq)}, bound max {kq.max()}"
    qa = (G["angle_mat"][kh, yh, xh] & 0xFFFFFF).astype(np.int64)
    dqa = qa - r.q_angle[ok][hit].astype(np.int64)
    assert np.all(np.abs(dqa) * 90.0 / Q24 <= 1e-4)
    _report({"label": "raster G-buffer codes, small terrain W=640 K=5", "pixels": int(hit.sum()),
             "depth_code_diff": code_counts(dq), "depth_code_bound_max": int(kq.max()),
             "angle_code_diff": code_counts(dqa)})
    # most codes agree exactly or to one rounding step
    assert (np.abs(dq) <= 1).mean() > 0.9
    assert np.array_equal(G["angle_mat"][kh, yh, xh] >> 24, r.mat[ok][hit])
    assert np.array_equal(G["inst"][kh, yh, xh], r.inst[ok][hit])
    assert np.all(G["depth"][kh, yh, xh] < 0xFFFFFF)
    assert np.all(G["depth"][k[~hit], y[~hit], x[~hit]] == 0xFFFFFF)


def test_raster_empty_scene_and_steep_beams(L):
    """An empty scene returns nothing; beams steeper than a camera's half
    field project outside its rows and return nothing."""
    w = synth.small_terrain(seed=6, n_frames=1, n_az=64)
    empty = synth.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32), np.zeros(0, np.uint16),
                        np.zeros(0, np.uint32))
    we = synth.Workload("empty", empty, w.sensors, w.frames, w.params, w.seed)
    g, _ = gpu_raster(L, we, 256, 6)
    assert not g["valid"].any() and np.all(g["tri"] == 0xFFFFFFFF)
    # 32-channel sensor spans -16..+15 deg; with K = 12 cameras (30 deg field)
    # the beams beyond +-15 deg at the image centre column cannot be read
    g2, _ = gpu_raster(L, w, 256, 12)
    T = oracle.build_tables(w.params)
    r = oracle.raster(w.scene, w.sensors, w.frames, T, w.seed, 256, 12)
    assert r.outside.any()
    assert np.all(g2["tri"][r.outside != 0] == 0xFFFFFFFF) and not g2["valid"][r.outside != 0].any()


def test_raster_rejects_bad_configurations(L):
    from paper_2208_10295_gb300 import capi
    w = synth.small_terrain(seed=6, n_frames=1, n_az=64)
    scene, _ = setup(L, w)
    beams = L.alloc_beams(L.total_beams(w.frames), FIELDS)
    for width, k in ((0, 6), (20000, 6), (256, 2), (256, 65)):
        with pytest.raises(capi.LidarError) as e:
            L.raster_cast_into(scene, w.frames, w.seed, beams, width=width, n_cameras=k)
        assert e.value.status == capi.LIDAR_EINVAL
