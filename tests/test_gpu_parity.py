"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small workloads are compared on every beam; the full-size workloads on
seeded samples of beams the oracle computes one by one, with the GPU run at
full size in the launch configuration the benchmark uses."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import frame_offsets, gpu_cast, oracle_cast, pick, setup, stratified_sample
from parity import compare, compare_subray, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REPORT = os.environ.get("LIDAR_PARITY_REPORT")


def _report(rep):
    print(json.dumps(rep))
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps(rep) + "\n")


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


def test_beam_dirs_match_oracle_bitwise(L):
    w = synth.cfg1()
    L.set_sensor(0, w.sensors[0])
    got = L.beam_dirs(0)
    want = oracle.beam_dirs(w.sensors[0].az_rad, w.sensors[0].el_rad)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_tables_match_oracle(L):
    w = synth.cfg1()
    T = L.build_tables(torch.tensor(w.params, device=L.device)).cpu().numpy().astype(np.float64)
    ref = oracle.build_tables(w.params)
    assert np.allclose(T, ref, rtol=2e-6, atol=2e-7)
    G = np.random.default_rng(0).normal(size=ref.shape)
    gp = L.build_tables_backward(torch.tensor(w.params, device=L.device),
                                 torch.tensor(G, dtype=torch.float32, device=L.device)).cpu().numpy()
    gref = oracle.build_tables_backward(w.params, G.astype(np.float32).astype(np.float64))
    assert np.allclose(gp, gref, rtol=1e-5, atol=1e-5 * np.abs(gref).max())


def test_cfg0_every_beam(L):
    w = synth.cfg0()
    gpu, _ = gpu_cast(L, w)
    ref = oracle_cast(w)
    rep = compare(gpu, ref, label="cfg0 all beams")
    _report(rep)
    assert rep["returns"] > 5000
    assert rep["exempt"] <= 0.01 * rep["beams"]


@pytest.mark.parametrize("seed", [77, 78])
def test_small_terrain_every_beam(L, seed):
    w = synth.small_terrain(seed=seed, n_frames=3, n_az=256)
    gpu, _ = gpu_cast(L, w)
    ref = oracle_cast(w)
    rep = compare(gpu, ref, label=f"small terrain seed {seed}, all beams of 3 frames")
    _report(rep)
    assert rep["exempt"] <= 0.02 * rep["beams"]


def test_small_terrain_range_exponent(L):
    w = synth.small_terrain(seed=5, n_frames=1, n_az=128, range_exp=2.0)
    gpu, _ = gpu_cast(L, w)
    ref = oracle_cast(w)
    _report(compare(gpu, ref, label="small terrain, I ~ 1/R^2"))


@pytest.mark.parametrize("n_subrays", [7, 3, 8])
def test_small_terrain_subrays(L, n_subrays):
    w = synth.small_terrain(seed=9, n_frames=2, n_az=128, n_subrays=n_subrays, divergence=2e-3)
    gpu, _ = gpu_cast(L, w)
    ref = oracle_cast(w)
    _report(compare_subray(gpu, ref, label=f"small terrain, {n_subrays} sub-rays"))


def test_cfg1_full_frame_every_beam(L):
    """The headline frame (262,144 beams over 1,036,288 triangles), every beam
    against the oracle's brute force (about 3.5 minutes of oracle time on 16
    host cores), the GPU on the benchmark's tree, in its launch shape, with
    its per-beam cost-bucket schedule measured on a pose 1.1 m away."""
    from bench import HEADLINE_LAUNCH, build_cfg1
    w = synth.cfg1()
    scene = build_cfg1(L, w)
    cfg0 = L.launch_config()
    try:
        L.set_launch_config(ray_order=1, **{k: v[0] for k, v in HEADLINE_LAUNCH.items()})
        setup(L, w, scene)
        near = w.frames.copy()
        near[0]["pose"][3] += 1.0
        near[0]["pose"][7] += 0.5
        L.schedule_by_cost(scene, near, w.seed, mode=1)
        beams = L.alloc_beams(L.total_beams(w.frames))
        L.cast_into(scene, w.frames, w.seed, beams)
        assert L.sync_status() == 0
        gpu = to_numpy(beams)
    finally:
        L.reset_schedule(0)
        L.set_launch_config(**cfg0)
    ref = oracle_cast(w)
    rep = compare(gpu, ref, label="cfg1 full frame, every beam")
    _report(rep)
    assert rep["beams"] == 262144
    # exemptions stay a small, counted minority (0.12 % measured: beams within
    # the edge band of a triangle, and depth ties where objects meet the terrain)
    assert rep["exempt"] <= 2e-3 * rep["beams"]
    # whole-frame properties that hold at any size
    v = gpu["valid"] != 0
    assert v.sum() > 50000
    assert np.all((gpu["range"][v] >= 0.5) & (gpu["range"][v] <= 200.0))
    assert np.all(gpu["intensity"][v] > 0)
    tri = gpu["tri"]
    hit = tri != 0xFFFFFFFF
    assert np.all(tri[hit] < w.scene.n_tris)
    assert np.array_equal(gpu["inst"][hit], w.scene.inst[tri[hit]])
    assert np.array_equal(gpu["mat"][hit], w.scene.mat[tri[hit]])
    assert np.all(np.isinf(gpu["t"][~hit]))


def test_cfg2_batched_sampled(L):
    from bench import build_cfg1  # the benchmark's hierarchy of the 1M-triangle scene
    w = synth.cfg2()
    gpu, _ = gpu_cast(L, w, scene=build_cfg1(L, w),
                      fields=("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst"))
    samples = stratified_sample(w, 4096, seed=2)
    ref = oracle_cast(w, samples)
    _report(compare(pick(gpu, w, samples), ref, label="cfg2 8 sensors x 64 frames, 4096 sampled beams"))


@pytest.mark.parametrize("n_subrays", [1, 7, 3])
def test_ray_order_and_launch_shapes_bit_identical(L, n_subrays):
    """Ray order, launch shape, traversal variant and cost schedule change
    timing only.  With several sub-rays per beam a beam's sub-rays run on
    neighbouring lanes (7: four beams per warp step, 3: ten), checked here
    with every traversal, the warp-synchronous one included."""
    w = synth.small_terrain(seed=3, n_frames=2, n_az=256, n_subrays=n_subrays,
                            divergence=2e-3 if n_subrays > 1 else 0.0)
    base, scene = gpu_cast(L, w)
    cfg0 = L.launch_config()
    try:
        for cfg in ({"ray_order": 0}, {"block_threads": 64, "tile_rays": 64}, {"traversal": 1}, {"traversal": 2},
                    {"traversal": 3}, {"traversal": 3, "block_threads": 128, "blocks_per_sm": 4},
                    {"block_threads": 256, "tile_rays": 512, "blocks_per_sm": 2},
                    {"block_threads": 256, "blocks_per_sm": 3}, {"block_threads": 128, "blocks_per_sm": 6},
                    {"block_threads": 256, "blocks_per_sm": 4, "traversal": 2}):
            L.set_launch_config(**cfg)
            other, _ = gpu_cast(L, w, scene)
            for k in base:
                assert np.array_equal(base[k].view(np.uint8), other[k].view(np.uint8)), (cfg, k)
        # the cost-ordered schedule changes timing only
        L.set_launch_config(**cfg0)
        for mode in (0, 1):
            L.schedule_by_cost(scene, w.frames[:1], w.seed, mode=mode)
            other, _ = gpu_cast(L, w, scene)
            for k in base:
                assert np.array_equal(base[k].view(np.uint8), other[k].view(np.uint8)), ("cost schedule", mode, k)
    finally:
        L.set_launch_config(**cfg0)
        L.reset_schedule(0)


@pytest.mark.parametrize("fused,block_threads", [(0, 128), (1, 64), (1, 256)])
def test_points_compaction_matches_dense(L, fused, block_threads):
    # 250 azimuths: frames end inside compaction tiles and the last tile is ragged
    w = synth.small_terrain(seed=4, n_frames=3, n_az=250)
    scene, _ = setup(L, w)
    n = L.total_beams(w.frames)
    assert n % 1024 != 0
    cfg0 = L.launch_config()
    L.set_launch_config(fused_scatter=fused, block_threads=block_threads)
    try:
        _check_points(L, w, scene, n)
    finally:
        L.set_launch_config(**cfg0)


def _check_points(L, w, scene, n):
    beams, pts = L.cast(scene, w.frames, w.seed, dense=True, points_capacity=n)
    assert L.sync_status() == 0
    g = to_numpy(beams)
    cnt = int(pts["count"].item())
    v = np.flatnonzero(g["valid"])
    assert cnt == v.size
    off = frame_offsets(w)
    fidx = np.searchsorted(off, v, side="right") - 1
    assert np.array_equal(pts["frame"][:cnt].cpu().numpy(), fidx)
    assert np.array_equal(pts["beam"][:cnt].cpu().numpy(), v - off[fidx])
    assert np.array_equal(pts["range"][:cnt].cpu().numpy(), g["range"][v])
    assert np.array_equal(pts["intensity"][:cnt].cpu().numpy(), g["intensity"][v])
    assert np.array_equal(pts["instance"][:cnt].cpu().numpy().view(np.uint32), g["inst"][v])
    dirs = L.beam_dirs(0)
    xyz = pts["xyz"][:cnt].cpu().numpy()
    assert np.allclose(xyz, g["range"][v, None] * dirs[v - off[fidx]], rtol=1e-6, atol=1e-6)
    # capacity overflow: count reports the need, nothing beyond capacity is written
    cap = cnt // 2
    pts2 = L.alloc_points(cap + 1)
    sentinel = torch.full((1,), -7.0, device=L.device)
    pts2["range"][cap:] = sentinel
    pts2 = {k: (v_[:cap] if k != "count" else v_) for k, v_ in pts2.items()}
    L.cast_into(scene, w.frames, w.seed, None, pts2)
    from paper_2208_10295_gb300 import capi
    assert L.sync_status() == capi.LIDAR_ECAPACITY
    assert int(pts2["count"].item()) == cnt


def test_empty_and_single_triangle_scenes(L):
    w = synth.small_terrain(seed=6, n_frames=1, n_az=64)
    empty = synth.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32), np.zeros(0, np.uint16),
                        np.zeros(0, np.uint32))
    we = synth.Workload("empty", empty, w.sensors, w.frames, w.params, w.seed)
    gpu, _ = gpu_cast(L, we)
    assert np.all(gpu["tri"] == 0xFFFFFFFF) and not gpu["valid"].any()
    one = synth.Scene(np.array([[-50, -50, -0.5], [50, -50, -0.5], [0, 80, -0.5]], np.float32) +
                      w.frames[0]["pose"][[3, 7, 11]],
                      np.array([[0, 1, 2]], np.uint32), np.array([1], np.uint16), np.array([42], np.uint32))
    w1 = synth.Workload("one", one, w.sensors, w.frames, w.params, w.seed)
    gpu, _ = gpu_cast(L, w1)
    ref = oracle_cast(w1)
    rep = compare(gpu, ref, label="single triangle")
    assert rep["hits"] > 100


@pytest.mark.parametrize("method", [0, 1])
def test_lbvh_invariants(L, method):
    """Both hierarchies (Karras LBVH, PLOC clustering): every leaf once, every
    node but the root once, parent boxes equal to their children's boxes, depth
    within the traversal stack."""
    w = synth.small_terrain(seed=8, n_cells=48, half=24.0, n_objects=20, n_frames=1, n_az=32)
    L.set_build_options(method=method)
    try:
        scene, _ = setup(L, w)
    finally:
        L.set_build_options(method=1)
    nodes, leaf_tri = scene.export()
    n = w.scene.n_tris
    assert nodes.shape[0] == n - 1
    assert np.array_equal(np.sort(leaf_tri), np.arange(n))
    child = nodes[:, 12:14].view(np.int32)
    seen_leaf = np.zeros(n, int)
    seen_node = np.zeros(n - 1, int)
    V = w.scene.verts[w.scene.tris[leaf_tri]]          # leaf-ordered triangles
    lo_t, hi_t = V.min(1), V.max(1)

    def box_of(c):
        if c < 0:
            return lo_t[~c], hi_t[~c]
        b = nodes[c]
        lo = np.minimum([b[0], b[2], b[8]], [b[4], b[6], b[10]])
        hi = np.maximum([b[1], b[3], b[9]], [b[5], b[7], b[11]])
        return lo, hi

    for i in range(n - 1):
        b = nodes[i]
        for side, c in enumerate(child[i]):
            if c < 0:
                seen_leaf[~c] += 1
            else:
                seen_node[c] += 1
            lo = np.array([b[0], b[2], b[8]] if side == 0 else [b[4], b[6], b[10]])
            hi = np.array([b[1], b[3], b[9]] if side == 0 else [b[5], b[7], b[11]])
            clo, chi = box_of(c)
            # the parent stores exactly the child's box (exact FP32 min/max)
            assert np.array_equal(lo, clo) and np.array_equal(hi, chi), (i, side)
    assert np.all(seen_leaf == 1)
    assert seen_node[0] == 0 and np.all(seen_node[1:] == 1)
    assert scene.info()["max_depth"] <= 96


@pytest.mark.parametrize("radius", [1, 16])
def test_ploc_tree_casts_bit_identical(L, radius):
    """The closest hit does not depend on the hierarchy: a PLOC tree gives every
    dense field bit for bit as the LBVH tree does (cfg0 and a small terrain
    with sub-rays), and its casts match the oracle."""
    for w in (synth.cfg0(), synth.small_terrain(seed=9, n_frames=2, n_az=128, n_subrays=7, divergence=2e-3)):
        L.set_build_options(method=0)
        try:
            base, _ = gpu_cast(L, w)
        finally:
            L.set_build_options(method=1)
        L.set_build_options(method=1, ploc_radius=radius)
        try:
            other, _ = gpu_cast(L, w)
        finally:
            L.set_build_options(method=1, ploc_radius=16)
        for k in base:
            assert np.array_equal(base[k].view(np.uint8), other[k].view(np.uint8)), (w.name, radius, k)


def test_ploc_cfg1_full_frame_bit_identical(L):
    w = synth.cfg1()
    fields = ("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst", "theta_deg")
    L.set_build_options(method=0)
    try:
        base, s0 = gpu_cast(L, w, fields=fields)
    finally:
        L.set_build_options(method=1)
    v0 = L.count_work(s0, w.frames, w.seed)["node_visits"]
    other, s1 = gpu_cast(L, w, fields=fields)
    v1 = L.count_work(s1, w.frames, w.seed)["node_visits"]
    for k in fields:
        assert np.array_equal(base[k].view(np.uint8), other[k].view(np.uint8)), k
    _report({"label": "cfg1 PLOC vs LBVH node fetches per ray", "lbvh": v0 / 262144, "ploc": v1 / 262144})


def _wide_tree_invariants(nodes, width, n_tris, lo_t, hi_t):
    """Every leaf once, every wide node but the root once (breadth-first: a
    child's slot is above its parent's), each child box equal to the union of
    the boxes below it (exact FP32 min/max), empty slots empty, internal
    children first with consecutive ids and the metadata that says so."""
    G = width // 4
    n = nodes.shape[0]
    f4 = nodes.reshape(n, 8 * G, 4)
    lo = np.stack([f4[:, (2 * a) * G:(2 * a) * G + G].reshape(n, width) for a in range(3)], -1)
    hi = np.stack([f4[:, (2 * a + 1) * G:(2 * a + 1) * G + G].reshape(n, width) for a in range(3)], -1)
    code = f4[:, 6 * G:7 * G].reshape(n, width).view(np.int32)
    # metadata: first internal child's id, mask of leaf slots; internal
    # children fill the first slots with consecutive ids
    meta = f4[:, 7 * G].view(np.int32)
    assert np.all(meta[:, 2:] == 0) and np.all(f4[:, 7 * G + 1:] == 0)
    for i in range(n):
        internal = code[i] > 0
        m = int(internal.sum())
        assert np.all(internal[:m]) and not internal[m:].any(), i
        assert np.array_equal(code[i, :m], meta[i, 0] + np.arange(m)), i
        leaf_bits = sum(1 << j for j in range(width) if code[i, j] < 0)
        assert meta[i, 1] == leaf_bits, i
    seen_leaf = np.zeros(n_tris, int)
    seen_node = np.zeros(n, int)
    box_lo = np.full((n, 3), np.inf, np.float32)
    box_hi = np.full((n, 3), -np.inf, np.float32)
    for i in range(n - 1, -1, -1):
        for j in range(width):
            c = int(code[i, j])
            empty = np.all(lo[i, j] == np.inf) and np.all(hi[i, j] == -np.inf)
            if empty:
                assert c == 0
                continue
            if c < 0:
                seen_leaf[~c] += 1
                want_lo, want_hi = lo_t[~c], hi_t[~c]
            else:
                assert i < c < n
                seen_node[c] += 1
                want_lo, want_hi = box_lo[c], box_hi[c]
            assert np.array_equal(lo[i, j], want_lo) and np.array_equal(hi[i, j], want_hi), (i, j)
            box_lo[i] = np.minimum(box_lo[i], lo[i, j])
            box_hi[i] = np.maximum(box_hi[i], hi[i, j])
    assert np.all(seen_leaf == 1)
    assert seen_node[0] == 0 and np.all(seen_node[1:] == 1)


@pytest.mark.parametrize("method,collapse", [(0, 0), (1, 0), (1, 1)])
def test_wide_tree_invariants(L, method, collapse):
    """The 4- and 8-wide trees collapsed from either binary hierarchy, by the
    largest-area rule or the SAH dynamic program, hold every leaf once with
    exact boxes; the 8-wide tree is shallower."""
    w = synth.small_terrain(seed=8, n_cells=48, half=24.0, n_objects=20, n_frames=1, n_az=32)
    L.set_build_options(method=method, collapse=collapse)
    try:
        scene, _ = setup(L, w)
    finally:
        L.set_build_options(method=1, collapse=0)
    _, leaf_tri = scene.export()
    V = w.scene.verts[w.scene.tris[leaf_tri]]
    lo_t, hi_t = V.min(1).astype(np.float32), V.max(1).astype(np.float32)
    info = scene.info()
    assert info["n_nodes8"] > 0 and info["levels8"] < info["levels4"]
    for width in (4, 8):
        _wide_tree_invariants(scene.export_wide(width), width, w.scene.n_tris, lo_t, hi_t)


def test_wide8_cfg1_full_frame_bit_identical(L):
    """The 8-wide traversal returns every dense field of the full cfg1 frame bit
    for bit as the 4-wide one, with fewer node fetches."""
    w = synth.cfg1()
    fields = ("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst", "theta_deg")
    cfg0 = L.launch_config()
    try:
        L.set_launch_config(traversal=2)
        base, scene = gpu_cast(L, w, fields=fields)
        c4 = L.count_work(scene, w.frames, w.seed)
        L.set_launch_config(traversal=3)
        other, _ = gpu_cast(L, w, scene, fields=fields)
        c8 = L.count_work(scene, w.frames, w.seed)
    finally:
        L.set_launch_config(**cfg0)
    for k in fields:
        assert np.array_equal(base[k].view(np.uint8), other[k].view(np.uint8)), k
    assert c8["node_bytes"] == 256 and c4["node_bytes"] == 128
    assert c8["node_visits"] < c4["node_visits"]
    _report({"label": "cfg1 node fetches per ray, 4-wide vs 8-wide", "wide4": c4["node_visits"] / 262144,
             "wide8": c8["node_visits"] / 262144, "tri_tests4": c4["tri_tests"] / 262144,
             "tri_tests8": c8["tri_tests"] / 262144})


def test_batch_and_graph_replay_match_direct_cast(L):
    """A captured batch (8-sensor rig, several frames) replays bit-identically
    to lidar_cast, and a pose update inside the graph matches a direct cast at
    the new poses."""
    w = synth.cfg2(n_frames=3)
    scene, _ = setup(L, w)
    n = L.total_beams(w.frames)
    fields = ("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst")
    direct = L.alloc_beams(n, fields)
    L.cast_into(scene, w.frames, w.seed, direct)
    B = L.batch(w.frames)
    got = L.alloc_beams(n, fields)
    B.cast_into(scene, w.seed, got)
    assert L.sync_status() == 0
    for k in fields:
        assert torch.equal(direct[k], got[k]), k
    # graph with a device pose buffer, replayed twice with different poses
    poses = torch.tensor(np.stack([f["pose"] for f in w.frames]), device=L.device)
    pts = L.alloc_points(n)
    G = B.graph(scene, w.seed, beams=got, points=pts, poses=poses)
    for shift in (0.0, 1.5):
        moved = w.frames.copy()
        for f in moved:
            f["pose"][3] += shift
        poses.copy_(torch.tensor(np.stack([f["pose"] for f in moved]), device=L.device))
        G.launch()
        ref = L.alloc_beams(n, fields)
        ref_pts = L.alloc_points(n)
        L.cast_into(scene, moved, w.seed, ref, ref_pts)
        assert L.sync_status() == 0
        for k in fields:
            assert torch.equal(ref[k], got[k]), (shift, k)
        c = int(ref_pts["count"].item())
        assert int(pts["count"].item()) == c
        assert torch.equal(ref_pts["range"][:c], pts["range"][:c])
    B.free()


def test_cfg4_city_subrays_sampled(L):
    """The 10.7M-triangle city, 7 sub-rays per beam, all 32 frames cast on the
    GPU; a seeded sample of beams is recomputed by the oracle (every sub-ray
    against every triangle)."""
    from bench import build_city  # the hierarchy the benchmark walks (PLOC + treelet rounds)
    w = synth.cfg4()
    gpu, _ = gpu_cast(L, w, scene=build_city(L, w),
                      fields=("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst", "sub"))
    samples = stratified_sample(w, 1280, seed=4)
    ref = oracle_cast(w, samples)
    rep = compare_subray(pick(gpu, w, samples), ref, label="cfg4 city, 7 sub-rays, 1280 sampled beams")
    rep["strict"] = rep["beams"] - rep["exempt"]
    _report(rep)
    # many hit beams have several sub-rays of near-equal intensity on the same
    # surface: those are checked through the ambiguous-choice path; the rest
    # (a unique strongest sub-ray, or a miss) are compared field by field
    assert rep["strict"] >= 300, rep


def test_direct_casts_back_to_back_with_reused_counters(L):
    """Direct casts alternate between two counter regions, each clearing the
    other for the next cast: a sequence of casts with and without a point
    cloud, of growing sizes (the regions are reallocated) and in both launch
    modes (fused scatter or not) reproduces the first cast's point cloud."""
    w = synth.small_terrain(seed=21, n_frames=1, n_az=256)
    big = synth.small_terrain(seed=22, n_frames=4, n_az=1024)
    scene, _ = setup(L, w)
    n = L.total_beams(w.frames)

    def points_of(frames, nb):
        pts = L.alloc_points(nb)
        L.cast_into(scene, frames, w.seed, None, pts)
        assert L.sync_status() == 0
        c = int(pts["count"].item())
        return c, {k: v[:c].clone() for k, v in pts.items() if k != "count"}

    c0, p0 = points_of(w.frames, n)
    assert c0 > 1000
    cfg0 = L.launch_config()
    try:
        for step in range(6):
            if step == 2:
                L.set_sensor(0, big.sensors[0])
                points_of(big.frames, L.total_beams(big.frames))   # larger: new regions
                L.set_sensor(0, w.sensors[0])
            if step == 4:
                L.set_launch_config(fused_scatter=0)
            dense = L.alloc_beams(n, ("valid",))
            L.cast_into(scene, w.frames, w.seed, dense)               # no point cloud
            assert L.sync_status() == 0
            assert int(dense["valid"].sum().item()) == c0
            c, p = points_of(w.frames, n)
            assert c == c0, step
            for k in p0:
                assert torch.equal(p[k], p0[k]), (step, k)
    finally:
        L.set_launch_config(**cfg0)


def test_degenerate_triangles_change_nothing(L):
    """Zero-area triangles (one point three times; two equal vertices and a
    third) appended to cfg0 on the beams' own paths, 5 and 12 m out: every
    dense field is bit for bit that of plain cfg0 (the original triangles keep
    their indices) and matches the oracle on every beam; none is ever hit."""
    w = synth.cfg0()
    base, _ = gpu_cast(L, w)
    dirs = L.beam_dirs(0).astype(np.float32)
    o = np.asarray(w.frames[0]["pose"], np.float32).reshape(3, 4)[:, 3]
    pick_b = np.arange(0, dirs.shape[0], 97)
    tris = []
    for s_ in (np.float32(5.0), np.float32(12.0)):
        p = o[None, :] + s_ * dirs[pick_b]
        tris += [[q, q, q] for q in p]
        tris += [[q, q, q + np.float32([0.0, 0.0, 2.0])] for q in p]
    v0 = w.scene.verts.shape[0]
    k = len(tris)
    sc = synth.Scene(np.concatenate([w.scene.verts, np.asarray(tris, np.float32).reshape(-1, 3)]),
                     np.concatenate([w.scene.tris, (v0 + np.arange(3 * k, dtype=np.uint32)).reshape(k, 3)]),
                     np.concatenate([w.scene.mat, np.zeros(k, np.uint16)]),
                     np.concatenate([w.scene.inst, np.full(k, 999, np.uint32)]))
    wd = synth.Workload("cfg0_degenerate", sc, w.sensors, w.frames, w.params, w.seed)
    got, _ = gpu_cast(L, wd)
    for key in base:
        assert np.array_equal(base[key].view(np.uint8), got[key].view(np.uint8)), key
    hit = got["tri"] != 0xFFFFFFFF
    assert np.all(got["tri"][hit] < w.scene.n_tris)
    _report(compare(got, oracle_cast(wd), label=f"cfg0 + {k} degenerate triangles on beam paths, every beam"))


def _sixteen_sensor_workload():
    """Every sensor slot filled, with what varies between sensors varying:
    spinning 16/32-channel and raster patterns whose beam counts are not
    multiples of 32, 1..8 sub-rays, noise with and without the range term,
    range exponent, gain, range limits and Eq. 5 constants.  Two frames per
    slot at different poses, the frame records in a shuffled slot order."""
    base = synth.small_terrain(seed=41, n_frames=4)
    rng = np.random.default_rng(4141)
    sensors = []
    for s in range(16):
        ns = 1 + s % 8
        kw = dict(r_min=float(rng.uniform(0.3, 1.0)), r_max=float(rng.uniform(25.0, 40.0)),
                  d_max=float(rng.uniform(20.0, 45.0)), RL_max=float(rng.uniform(0.2, 0.9)),
                  sigma=float(rng.choice([0.0, 0.01, 0.03])), sigma_k=float(rng.choice([0.0, 0.002])),
                  gain=float(rng.uniform(0.5, 2.0)), range_exp=float(rng.choice([0.0, 2.0])),
                  n_subrays=ns, divergence_rad=2e-3 if ns > 1 else 0.0)
        if s % 3 == 0:
            spec = synth.sensors.sensor_16ch(int(rng.integers(40, 90)), **kw)
        elif s % 3 == 1:
            spec = synth.sensors.sensor_32ch(int(rng.integers(20, 45)), **kw)
        else:
            spec = synth.sensors.sensor_raster(int(rng.integers(20, 40)), int(rng.integers(9, 23)),
                                               fov_h=100.0, fov_v=30.0, **kw)
        sensors.append(spec)
    poses = base.frames["pose"]
    entries = []
    for k, s in enumerate(rng.permutation(np.repeat(np.arange(16), 2))):
        entries.append((int(s), 100 + k, poses[k % len(poses)]))
    return synth.Workload("sixteen_sensors", base.scene, sensors, synth.workloads.make_frames(entries),
                          base.params, base.seed)


def test_all_sensor_slots_mixed_batch_every_beam(L):
    """One cast over frames of all 16 sensor slots (the most the context
    holds), mixed sub-ray counts and sensor constants, ragged beam counts:
    every beam against the oracle, and the point cloud in (frame, beam) order
    against the dense output."""
    w = _sixteen_sensor_workload()
    assert len(w.sensors) == 16
    gpu, scene = gpu_cast(L, w)
    ref = oracle_cast(w)
    gmax = max(s.gain for s in w.sensors)
    rep = compare_subray(gpu, ref, gain=gmax, label=f"16 sensor slots, 32 frames, {len(gpu['valid'])} beams, 1-8 sub-rays")
    _report(rep)
    assert rep["returns"] > 1000
    beams, points = L.cast(scene, w.frames, w.seed, points_capacity=L.total_beams(w.frames))
    n = int(points["count"].item())
    v = np.flatnonzero(gpu["valid"] != 0)
    assert n == v.size
    assert np.array_equal(points["range"][:n].cpu().numpy().view(np.uint32), gpu["range"][v].view(np.uint32))
    assert np.array_equal(points["intensity"][:n].cpu().numpy().view(np.uint32), gpu["intensity"][v].view(np.uint32))
    scene.free()


def _box_tris(lo, hi):
    """12 triangles (outward winding) of the axis-aligned box [lo, hi]."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], np.float32)
    f = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6], [4, 6, 7], [0, 1, 5], [0, 5, 4],
                  [1, 2, 6], [1, 6, 5], [2, 3, 7], [2, 7, 6], [3, 0, 4], [3, 4, 7]], np.uint32)
    return v, f


def _in_plane_workload():
    """Beams lying exactly in box planes.  The sensor sits at (0, 0, 1); its
    horizontal beams (elevation 0: direction z exactly 0) run in the plane
    z = 1, which is the top of some boxes and the bottom of others, and its
    azimuth-0 beams (direction y exactly 0) run in the plane y = 0, a face of
    some boxes.  Their slab distances there are 0 * inf = NaN, which the box
    test must ignore (the axis is then unconstrained) in the leaves' boxes and
    in every union box above them.  Four walls close the arena so every
    horizontal beam ends on a surface."""
    rng = np.random.default_rng(5150)
    verts, tris = [], []

    def add(v, f):
        tris.append(f + sum(len(x) for x in verts))
        verts.append(v)
    add(np.array([[-40, -40, 0], [40, -40, 0], [40, 40, 0], [-40, 40, 0]], np.float32),
        np.array([[0, 1, 2], [0, 2, 3]], np.uint32))
    for lo, hi in (((30, -40, 0), (31, 40, 6)), ((-31, -40, 0), (-30, 40, 6)),
                   ((-40, 30, 0), (40, 31, 6)), ((-40, -31, 0), (40, -30, 6))):
        add(*_box_tris(lo, hi))
    for k in range(40):
        x0 = float(rng.integers(3, 25)) * (1 if k % 2 else -1)
        y0 = 0.0 if k % 5 == 0 else float(rng.integers(-25, 25))
        sx, sy = float(rng.integers(1, 4)), float(rng.integers(1, 4))
        z0, z1 = (0.0, 1.0) if k % 3 == 0 else ((1.0, 2.5) if k % 3 == 1 else (0.0, float(rng.integers(2, 4))))
        add(*_box_tris((x0, y0, z0), (x0 + sx, y0 + sy, z1)))
    V = np.concatenate(verts)
    T = np.concatenate(tris)
    n = T.shape[0]
    scene = synth.Scene(V, T, (np.arange(n) % 2).astype(np.uint16), (1 + np.arange(n) // 12).astype(np.uint32))
    el = np.array([-10.0, -1.0, 0.0, 1.0, 10.0])
    az, elv = synth.sensors.spinning_pattern(el, 720)
    sensor = synth.SensorSpec("in_plane", az, elv, r_min=0.3, r_max=80.0, d_max=80.0, RL_max=0.5, sigma=0.0)
    frames = synth.workloads.make_frames([(0, 0, synth.workloads.pose_rows(np.eye(3), [0.0, 0.0, 1.0]))])
    params = synth.material_params(np.random.default_rng(5151), 2)
    return synth.Workload("in_plane", scene, [sensor], frames, params, 77)


def test_beams_lying_in_box_planes(L):
    """Beams in the planes of box faces (NaN slab distances): every traversal
    (binary per lane, warp-synchronous, 4-wide and 8-wide, whose box tests take
    the near and far distances by different min/max sequences) gives the same
    records bit for bit, and they match the oracle's brute force on every beam
    outside the counted exemptions."""
    w = _in_plane_workload()
    d = w.sensors[0]
    dirs = None
    cfg0 = L.launch_config()
    try:
        L.set_launch_config(traversal=2)
        base, scene = gpu_cast(L, w)
        dirs = L.beam_dirs(0)
        for tv in (0, 1, 3):
            L.set_launch_config(traversal=tv)
            other, _ = gpu_cast(L, w, scene)
            for k in base:
                assert np.array_equal(base[k].view(np.uint8), other[k].view(np.uint8)), (tv, k)
    finally:
        L.set_launch_config(**cfg0)
    # the premise: exact zeros in the directions of the in-plane beams
    horiz = d.el_rad == 0.0
    assert np.all(dirs[horiz, 2] == 0.0) and np.all(dirs[d.az_rad == 0.0, 1] == 0.0)
    ref = oracle_cast(w)
    rep = compare(base, ref, label=f"beams in box planes, {d.n_beams} beams")
    _report(rep)
    assert np.all(base["tri"][horiz] != 0xFFFFFFFF)
    # every beam up to +1 deg ends on a surface (the +10 deg channel clears the 6 m walls)
    low = d.el_rad < np.deg2rad(5.0)
    assert np.all(ref["tri"][low] != 0xFFFFFFFF) and np.all(base["tri"][low] != 0xFFFFFFFF)
    scene.free()


def test_points_download(L):
    """lidar_points_download copies the first `count` points of every field
    present on both sides (pinned host tensors, a side stream) bit for bit as
    the device holds them, leaves the rest of the host buffers alone, skips
    fields missing on either side, and rejects a count above a capacity."""
    w = synth.small_terrain(seed=12, n_frames=2, n_az=200)
    scene, _ = setup(L, w)
    n = L.total_beams(w.frames)
    _, pts = L.cast(scene, w.frames, w.seed, dense=False, points_capacity=n)
    assert L.sync_status() == 0
    cnt = int(pts["count"].item())
    assert 0 < cnt < n
    host = {k: torch.full(v.shape, 0x5A, dtype=v.dtype, pin_memory=True) for k, v in pts.items()}
    del host["normal"]
    s = torch.cuda.Stream(device=L.device)
    s.wait_stream(L.stream)
    L.download_points(pts, host, cnt, stream=s)
    s.synchronize()
    for k, h in host.items():
        if k == "count":
            continue
        d = pts[k].cpu()
        assert torch.equal(h[:cnt], d[:cnt]), k
        assert bool((h[cnt:] == 0x5A).all()), k
    L.download_points(pts, host, 0)
    from paper_2208_10295_gb300 import capi
    for bad in (n + 1, -1):
        with pytest.raises(capi.LidarError) as e:
            L.download_points(pts, host, bad)
        assert e.value.status == capi.LIDAR_EINVAL
    scene.free()


def _points_np(p):
    c = int(p["count"].item())
    return c, {k: v[:c].cpu().numpy() for k, v in p.items() if k != "count"}


def test_overlapped_direct_casts_match_serial(L):
    """Consecutive direct casts whose outputs share no memory may overlap (the
    next cast starts on the SMs the previous one's last traversals leave idle).
    Six casts of three frames in rotation into three sets of buffers, with no
    synchronisation between them (one of the repeat casts writes no dense
    records), give bit for bit what casts one after the other give; so do
    back-to-back casts of different frames into the same buffers (those the
    library orders one after the other)."""
    w = synth.small_terrain(seed=23, n_frames=3, n_az=512)
    scene, _ = setup(L, w)
    nb = w.sensors[0].n_beams
    frames = [w.frames[k:k + 1] for k in range(3)]
    fields = ("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst")
    assert L.cast_overlap()
    try:
        L.set_cast_overlap(False)
        ref = []
        for k in range(3):
            d, p = L.alloc_beams(nb, fields), L.alloc_points(nb)
            L.cast_into(scene, frames[k], w.seed, d, p)
            assert L.sync_status() == 0
            ref.append((to_numpy(d), _points_np(p)))
        L.set_cast_overlap(True)
        bufs = [(L.alloc_beams(nb, fields), L.alloc_points(nb)) for _ in range(3)]
        for i in range(6):
            d, p = bufs[i % 3]
            L.cast_into(scene, frames[i % 3], w.seed, d if i % 3 != 1 or i < 3 else None, p)
        torch.cuda.synchronize()
        assert L.sync_status() == 0
        for k in range(3):
            d, p = bufs[k]
            gd = to_numpy(d)
            for f in fields:
                assert np.array_equal(gd[f].view(np.uint8), ref[k][0][f].view(np.uint8)), (k, f)
            c, pts = _points_np(p)
            assert c == ref[k][1][0], k
            for f in pts:
                assert np.array_equal(pts[f].view(np.uint8), ref[k][1][1][f].view(np.uint8)), (k, f)
        # the same buffers for every cast: each cast follows the one before it
        d, p = bufs[0]
        for k in (1, 2, 0, 2):
            L.cast_into(scene, frames[k], w.seed, d, p)
        torch.cuda.synchronize()
        assert L.sync_status() == 0
        gd = to_numpy(d)
        for f in fields:
            assert np.array_equal(gd[f].view(np.uint8), ref[2][0][f].view(np.uint8)), f
        c, pts = _points_np(p)
        assert c == ref[2][1][0]
        for f in pts:
            assert np.array_equal(pts[f].view(np.uint8), ref[2][1][1][f].view(np.uint8)), f
    finally:
        L.set_cast_overlap(True)
        scene.free()


def test_sah_collapse_casts_bit_identical(L):
    """The wide trees chosen by the SAH dynamic program give every dense field
    of the full cfg1 frame and of a small terrain with sub-rays bit for bit as
    the largest-area collapse does, with both wide traversals."""
    fields = ("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst", "theta_deg")
    cfg0 = L.launch_config()
    try:
        for w in (synth.cfg1(), synth.small_terrain(seed=9, n_frames=2, n_az=128, n_subrays=7, divergence=2e-3)):
            for tv in (2, 3):
                L.set_launch_config(traversal=tv)
                L.set_build_options(method=1, collapse=0)
                base, s0 = gpu_cast(L, w, fields=fields)
                L.set_build_options(method=1, collapse=1)
                other, s1 = gpu_cast(L, w, fields=fields)
                for k in fields:
                    assert np.array_equal(base[k].view(np.uint8), other[k].view(np.uint8)), (w.name, tv, k)
                assert s1.info()["n_nodes4"] <= s0.info()["n_nodes4"]
                s0.free()
                s1.free()
    finally:
        L.set_build_options(method=1, collapse=0)
        L.set_launch_config(**cfg0)


def test_overlapped_casts_of_many_frames(L):
    """Casts of more than four frames take their frame table through a copy on
    the stream (not the launch parameters); back to back into rotating buffers
    without synchronisation they still give every cast's point cloud bit for
    bit as casts one after the other do."""
    w = synth.small_terrain(seed=24, n_frames=6, n_az=256)
    scene, _ = setup(L, w)
    n = L.total_beams(w.frames)
    sets = [w.frames, w.frames[::-1].copy()]
    try:
        L.set_cast_overlap(False)
        ref = []
        for fr in sets:
            p = L.alloc_points(n)
            L.cast_into(scene, fr, w.seed, None, p)
            assert L.sync_status() == 0
            ref.append(_points_np(p))
        L.set_cast_overlap(True)
        bufs = [L.alloc_points(n) for _ in range(3)]
        order = [0, 1, 0, 1, 1, 0]
        for i, k in enumerate(order):
            L.cast_into(scene, sets[k], w.seed, None, bufs[i % 3])
        torch.cuda.synchronize()
        assert L.sync_status() == 0
        for j in range(3):
            k = order[3 + j]
            c, pts = _points_np(bufs[j])
            assert c == ref[k][0], j
            for f in pts:
                assert np.array_equal(pts[f].view(np.uint8), ref[k][1][f].view(np.uint8)), (j, f)
    finally:
        L.set_cast_overlap(True)
        scene.free()


def test_streaming_autotune_gives_the_same_points(L):
    """The tuner's streaming regime (back-to-back casts into rotating point
    buffers, no flush) picks a launch among the shapes the end-to-end loop
    allows; casts in it give the point cloud of the default launch bit for
    bit, one at a time and back to back."""
    from bench import STREAM_LAUNCH
    from paper_2208_10295_gb300.tune import autotune
    w = synth.small_terrain(seed=29, n_frames=1, n_az=512)
    scene, _ = setup(L, w)
    nb = w.sensors[0].n_beams
    cfg0 = L.launch_config()
    ref = L.alloc_points(nb)
    L.cast_into(scene, w.frames, w.seed, None, ref)
    assert L.sync_status() == 0
    c_ref, p_ref = _points_np(ref)
    try:
        cfg, ms = autotune(L, scene, w.frames, w.seed, points=True, streaming=True, restrict=STREAM_LAUNCH,
                           cache_path=None)
        assert cfg["block_threads"] == 256 and cfg["blocks_per_sm"] in (2, 3) and ms > 0
        bufs = [L.alloc_points(nb) for _ in range(3)]
        for k in range(6):
            L.cast_into(scene, w.frames, w.seed, None, bufs[k % 3])
        assert L.sync_status() == 0
        for b in bufs:
            c, p = _points_np(b)
            assert c == c_ref
            for f in p_ref:
                assert np.array_equal(p[f].view(np.uint8), p_ref[f].view(np.uint8)), f
    finally:
        L.set_launch_config(**cfg0)
        L.reset_schedule(0)
