"""GPU parity of rolling-shutter sweeps, multi-echo returns and range-scaled
noise against the oracle.

Dense outputs follow the ray-cast contract (tests/parity.py).  Echoes: count,
sub-ray index and triangle bit-exact outside the counted exemptions (EDGE,
TIE, CUTOFF of any sub-ray, and ECHO: a near-tie in intensity or range, or a
range gap within tolerance of the separation); echo range 1e-5 relative,
intensity 1e-4 relative."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_cast, oracle_cast, setup
from parity import compare, compare_subray, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REPORT = os.environ.get("LIDAR_PARITY_REPORT")
FLAG_ECHO = 32


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


def sweeps_of(w):
    """Consecutive trajectory poses as the start and end of each sweep."""
    fr = w.frames
    return synth.make_sweep_frames([(int(fr[k]["sensor"]), int(fr[k]["frame"]), fr[k]["pose"], fr[k + 1]["pose"])
                                    for k in range(len(fr) - 1)])


def gpu_sweep(L, w, sweeps, n_echoes, mode, sep, scene=None):
    scene, _ = setup(L, w, scene)
    n = L.total_beams(sweeps)
    beams = L.alloc_beams(n)
    echoes = L.alloc_echoes(n, n_echoes)
    L.cast_sweep_into(scene, sweeps, w.seed, beams, echoes, mode=mode, separation=sep)
    assert L.sync_status() == 0
    return to_numpy(beams), {k: v.cpu().numpy() for k, v in echoes.items()}, scene


def sweep_offsets(w, sweeps):
    nb = np.array([w.sensors[int(s)].n_beams for s in sweeps["sensor"]], np.int64)
    return np.concatenate([[0], np.cumsum(nb)[:-1]])


def compare_echoes(ge, r, label):
    flags = r.flags.astype(np.int64)
    ok = (flags & (1 | 2 | 4 | FLAG_ECHO)) == 0
    sub_bad = (r.sub_flags.astype(np.int64) & (1 | 2 | 4)).any(axis=1)
    ok &= ~sub_bad
    rep = {"label": label, "beams": int(flags.size), "echo_exempt": int((~ok).sum())}
    assert np.array_equal(ge["count"][ok], r.echo_count[ok]), f"{label}: echo count differs"
    ne = r.echo_range.shape[1]
    for j in range(ne):
        have = ok & (r.echo_count > j)
        assert np.array_equal(ge["sub"][have, j], r.echo_sub[have, j]), f"{label}: echo {j} sub-ray differs"
        assert np.array_equal(ge["tri"][have, j].view(np.uint32), r.echo_tri[have, j]), f"{label}: echo {j} tri"
        dr = np.abs(ge["range"][have, j] - r.echo_range[have, j]) / r.echo_range[have, j]
        dI = np.abs(ge["intensity"][have, j] - r.echo_intensity[have, j])
        assert np.all(dr <= 1e-5), f"{label}: echo {j} range"
        assert np.all(dI <= 1e-4 * np.abs(r.echo_intensity[have, j]) + 1e-7), f"{label}: echo {j} intensity"
        rep[f"echo{j}_present"] = int(have.sum())
    rep["multi_echo_beams"] = int((ok & (r.echo_count > 1)).sum())
    return rep


@pytest.mark.parametrize("mode,n_echoes,sep", [(0, 3, 0.5), (1, 2, 0.3)])
def test_sweep_small_terrain_every_beam(L, mode, n_echoes, sep):
    w = synth.small_terrain(seed=9, n_frames=3, n_az=128, n_subrays=7, divergence=2e-3)
    w.sensors[0].sigma_k = 0.01
    sw = sweeps_of(w)
    g, ge, _ = gpu_sweep(L, w, sw, n_echoes, mode, sep)
    T = oracle.build_tables(w.params)
    r = oracle.cast_sweep(w.scene, w.sensors, sw, T, w.seed, echoes=(n_echoes, mode, sep))
    _report(compare_subray(g, r, label=f"sweep small terrain, 7 sub-rays, sigma_k 0.01, echoes mode {mode}"))
    _report(compare_echoes(ge, r, f"echoes mode {mode} n={n_echoes} sep={sep}, small terrain every beam"))


def test_sweep_cfg1_trajectory_sampled(L):
    """Two full 262,144-beam sweeps along the cfg3 trajectory (the sensor moves
    about a metre per sweep) over the cfg1 scene."""
    w1 = synth.cfg1()
    w3 = synth.cfg3(n_frames=3)
    w = synth.Workload("sweep", w1.scene, w1.sensors, w3.frames, w1.params, w1.seed)
    sw = sweeps_of(w)
    g, ge, _ = gpu_sweep(L, w, sw, 2, 1, 0.5)
    # seeded sample over both sweeps
    rng = np.random.default_rng(11)
    sf = np.repeat(np.arange(len(sw)), 384)
    sb = np.concatenate([np.sort(rng.choice(w1.sensors[0].n_beams, 384, replace=False)) for _ in range(len(sw))])
    T = oracle.build_tables(w.params)
    r = oracle.cast_sweep(w.scene, w.sensors, sw, T, w.seed, samples=(sf, sb), echoes=(2, 1, 0.5))
    idx = sweep_offsets(w, sw)[sf] + sb
    gs = {k: v[idx] for k, v in g.items()}
    _report(compare(gs, r, label="sweep cfg1 trajectory, 2 x 262,144 beams, 768 sampled"))
    _report(compare_echoes({k: v[idx] for k, v in ge.items()}, r, "echoes first/last, cfg1 sweeps, 768 sampled"))
    # the motion matters: a static sweep at the start pose gives other ranges
    assert g["valid"].sum() > 100000


def test_range_scaled_noise_cast_every_beam(L):
    w = synth.small_terrain(seed=81, n_frames=2, n_az=256)
    w.sensors[0].sigma = 0.05
    w.sensors[0].sigma_k = 0.02
    gpu, _ = gpu_cast(L, w)
    _report(compare(gpu, oracle_cast(w), label="small terrain, noise 0.05 + 0.02 t"))


def test_sweep_rejects_bad_echo_arguments(L):
    from paper_2208_10295_gb300 import capi
    w = synth.small_terrain(seed=9, n_frames=2, n_az=64)
    sw = sweeps_of(w)
    scene, _ = setup(L, w)
    n = L.total_beams(sw)
    for ne, mode, sep in ((5, 0, 1.0), (2, 2, 1.0), (2, 0, -1.0), (2, 1, float("nan"))):
        echoes = L.alloc_echoes(n, ne)
        with pytest.raises(capi.LidarError) as e:
            L.cast_sweep_into(scene, sw, w.seed, None, echoes, mode=mode, separation=sep)
        assert e.value.status == capi.LIDAR_EINVAL


def test_sweep_records_independent_of_echoes_shape_and_schedule(L):
    """The sweep cast runs on persistent, scheduled warp tiles with or without
    echoes: its dense records are bit for bit the same with echoes requested or
    not, at three launch shapes, in beam or Morton order, with the cost
    schedule, and its echoes are the same at every shape."""
    w = synth.small_terrain(seed=12, n_frames=3, n_az=128, n_subrays=7, divergence=2e-3)
    sw = sweeps_of(w)
    scene, _ = setup(L, w)
    n = L.total_beams(sw)
    cfg0 = L.launch_config()
    base = L.alloc_beams(n)
    base_e = L.alloc_echoes(n, 2)
    L.cast_sweep_into(scene, sw, w.seed, base, base_e, mode=1, separation=0.5)
    assert L.sync_status() == 0
    try:
        for cfg in ({}, {"ray_order": 0}, {"block_threads": 128, "blocks_per_sm": 4},
                    {"block_threads": 64, "blocks_per_sm": 12}):
            L.set_launch_config(**cfg)
            for sched in (None, 1):
                if sched is not None:
                    L.schedule_by_cost(scene, w.frames[:1], w.seed, mode=sched)
                a = L.alloc_beams(n)
                L.cast_sweep_into(scene, sw, w.seed, a)
                b = L.alloc_beams(n)
                e = L.alloc_echoes(n, 2)
                L.cast_sweep_into(scene, sw, w.seed, b, e, mode=1, separation=0.5)
                assert L.sync_status() == 0
                for k in base:
                    assert torch.equal(a[k], base[k]), (cfg, sched, k)
                    assert torch.equal(b[k], base[k]), (cfg, sched, k)
                for k in base_e:
                    assert torch.equal(e[k], base_e[k]), (cfg, sched, k)
                L.reset_schedule(0)
    finally:
        L.set_launch_config(**cfg0)
        L.reset_schedule(0)
