"""Error paths of the C ABI on a GPU, none of which faults the device:
argument checks, calls in the wrong state, capacity overflow, and allocation
failures injected on the host (LIDAR_FAULT_ALLOC_AT, in a child process so
the allocation count starts from zero)."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_wrong_state_and_bad_arguments(L):
    from paper_2208_10295_gb300 import capi
    w = synth.small_terrain(seed=41, n_frames=1, n_az=64)
    scene = L.build_scene(w.scene.verts, w.scene.tris, w.scene.mat, w.scene.inst)
    # cast before any material table
    fresh = type(L)(0)
    s2 = fresh.build_scene(w.scene.verts, w.scene.tris, w.scene.mat, w.scene.inst)
    fresh.set_sensor(0, w.sensors[0])
    with pytest.raises(capi.LidarError) as e:
        fresh.cast(s2, w.frames, w.seed)
    assert e.value.status == capi.LIDAR_ESTATE
    fresh.close()
    # a frame that names an empty sensor slot
    L.set_sensor(0, w.sensors[0])
    L.set_materials(L.build_tables(torch.tensor(w.params, device=L.device)))
    out = L.alloc_beams(w.sensors[0].n_beams)
    bad = w.frames.copy()
    bad["sensor"] = 5
    with pytest.raises(capi.LidarError) as e:
        L.cast_into(scene, bad, w.seed, out)
    assert e.value.status == capi.LIDAR_ESTATE
    # non-finite pose
    bad = w.frames.copy()
    bad[0]["pose"][0] = np.nan
    with pytest.raises(capi.LidarError) as e:
        L.cast_into(scene, bad, w.seed, out)
    assert e.value.status == capi.LIDAR_EINVAL
    # invalid sensor descriptions
    s = synth.SensorSpec("x", np.zeros(4), np.zeros(4), r_min=5.0, r_max=1.0)
    with pytest.raises(capi.LidarError) as e:
        L.set_sensor(1, s)
    assert e.value.status == capi.LIDAR_EINVAL
    s = synth.SensorSpec("x", np.zeros(4), np.zeros(4), n_subrays=9)
    with pytest.raises(capi.LidarError):
        L.set_sensor(1, s)
    # invalid launch configurations
    for cfg in ({"block_threads": 48}, {"block_threads": 512}, {"tile_rays": 40}, {"traversal": 7}):
        with pytest.raises(capi.LidarError) as e:
            L.set_launch_config(**cfg)
        assert e.value.status == capi.LIDAR_EINVAL
    # out-of-range vertex index: rejected by the build, reported on the host
    tris = w.scene.tris.copy()
    tris[3, 1] = w.scene.verts.shape[0] + 10
    with pytest.raises(capi.LidarError) as e:
        L.build_scene(w.scene.verts, tris, w.scene.mat, w.scene.inst)
    assert e.value.status == capi.LIDAR_EINVAL
    # the context is still usable afterwards
    beams, _ = L.cast(scene, w.frames, w.seed)
    assert L.sync_status() == 0
    # a batch refuses to run after its sensor changed
    B = L.batch(w.frames)
    w2 = synth.small_terrain(seed=41, n_frames=1, n_az=32)
    L.set_sensor(0, w2.sensors[0])
    with pytest.raises(capi.LidarError) as e:
        B.cast_into(scene, w.seed, L.alloc_beams(beams["valid"].shape[0]))
    assert e.value.status == capi.LIDAR_ESTATE
    B.free()


_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import torch, synth
from paper_2208_10295_gb300 import Lidar, capi
w = synth.small_terrain(seed=42, n_frames=1, n_az=64)
codes = []
try:
    L = Lidar(0)
    scene = L.build_scene(w.scene.verts, w.scene.tris, w.scene.mat, w.scene.inst)
    L.set_sensor(0, w.sensors[0])
    L.set_materials(L.build_tables(torch.tensor(w.params, device="cuda")))
    L.cast(scene, w.frames, w.seed, points_capacity=1000)
    codes.append(L.sync_status())
except capi.LidarError as e:
    codes.append(e.status)
print("STATUS", codes[-1])
"""


@pytest.mark.parametrize("nth", [1, 2, 3, 4, 6])
def test_injected_allocation_failure(L, nth):
    """The n-th device allocation of a fresh process fails: the call that made
    it returns LIDAR_ENOMEM (or later calls report a clean state error), and
    nothing crashes."""
    from paper_2208_10295_gb300 import capi
    env = dict(os.environ, LIDAR_FAULT_ALLOC_AT=str(nth))
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    status = int(r.stdout.strip().split("STATUS")[-1])
    assert status in (capi.LIDAR_ENOMEM, capi.LIDAR_ECAPACITY, capi.LIDAR_OK), status
    if nth <= 3:
        assert status == capi.LIDAR_ENOMEM


def test_grid_wait_runs_out_and_recovers(L):
    """The bounded grid-wide wait of a cast with the point-cloud scatter fused
    into the cast kernel, made to run out: with a wait limit of 0 ns every
    block that arrives before the last one gives up at its first check, records
    LIDAR_ETIMEOUT and leaves the kernel (no hang, no fault).  The dense
    records, written before the wait, are intact; with the default limit
    restored the next cast reproduces the reference point cloud bit for bit."""
    from paper_2208_10295_gb300 import capi
    w = synth.small_terrain(seed=43, n_frames=4, n_az=1024)
    scene = L.build_scene(w.scene.verts, w.scene.tris, w.scene.mat, w.scene.inst)
    L.set_sensor(0, w.sensors[0])
    L.set_materials(L.build_tables(torch.tensor(w.params, device=L.device)))
    n = L.total_beams(w.frames)
    cfg0 = L.launch_config()
    limit0 = L.wait_limit()
    assert limit0 == 2_000_000_000
    try:
        # the grid-wide wait belongs to casts one after the other (an overlapped
        # cast compacts in a separate kernel, without that wait)
        L.set_cast_overlap(False)
        L.set_launch_config(fused_scatter=1)
        if not L.launch_config()["fused_scatter"]:
            pytest.skip("no cooperative launch on this device")
        ref_beams, ref_pts = L.cast(scene, w.frames, w.seed, dense=True, points_capacity=n)
        assert L.sync_status() == 0
        c0 = int(ref_pts["count"].item())
        assert c0 > 1000
        L.set_wait_limit(0)
        beams, _ = L.cast(scene, w.frames, w.seed, dense=True, points_capacity=n)
        assert L.sync_status() == capi.LIDAR_ETIMEOUT
        assert "timed out" in capi.last_error()
        for k in ref_beams:
            assert torch.equal(beams[k], ref_beams[k]), k
        L.set_wait_limit(limit0)
        _, pts = L.cast(scene, w.frames, w.seed, dense=False, points_capacity=n)
        assert L.sync_status() == 0
        assert int(pts["count"].item()) == c0
        for k in ref_pts:
            if k != "count":
                assert torch.equal(pts[k][:c0], ref_pts[k][:c0]), k
    finally:
        L.set_wait_limit(limit0)
        L.set_launch_config(**cfg0)
        L.set_cast_overlap(True)
        scene.free()
