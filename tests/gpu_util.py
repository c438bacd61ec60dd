"""Helpers for the GPU tests: run a workload through the C ABI and the oracle."""
import numpy as np
import pytest

import oracle
from parity import to_numpy

torch = pytest.importorskip("torch")


def frame_offsets(w):
    nb = np.array([w.sensors[int(s)].n_beams for s in w.frames["sensor"]], np.int64)
    return np.concatenate([[0], np.cumsum(nb)[:-1]])


def setup(L, w, scene=None):
    if scene is None:
        scene = L.build_scene(w.scene.verts, w.scene.tris, w.scene.mat, w.scene.inst)
    for s, spec in enumerate(w.sensors):
        L.set_sensor(s, spec)
    table = L.build_tables(torch.tensor(w.params, device=L.device))
    L.set_materials(table)
    return scene, table


def gpu_cast(L, w, scene=None, fields=None):
    scene, table = setup(L, w, scene)
    n = L.total_beams(w.frames)
    beams = L.alloc_beams(n) if fields is None else L.alloc_beams(n, fields)
    L.cast_into(scene, w.frames, w.seed, beams)
    st = L.sync_status()
    assert st == 0, f"device status {st}"
    return to_numpy(beams), scene


def stratified_sample(w, n, seed=0):
    """Seeded sample of (frame entry, beam) pairs spread over frames and sensors."""
    rng = np.random.default_rng(seed)
    F = len(w.frames)
    per = max(1, n // F)
    sf, sb = [], []
    for k in range(F):
        nb = w.sensors[int(w.frames[k]["sensor"])].n_beams
        m = min(per, nb)
        sf.append(np.full(m, k, np.int64))
        sb.append(np.sort(rng.choice(nb, m, replace=False)).astype(np.int64))
    sf = np.concatenate(sf)
    sb = np.concatenate(sb)
    if sf.size > n:
        keep = np.sort(rng.choice(sf.size, n, replace=False))
        sf, sb = sf[keep], sb[keep]
    return sf, sb


def oracle_cast(w, samples=None, table=None):
    T = oracle.build_tables(w.params) if table is None else table
    return oracle.cast(w.scene, w.sensors, w.frames, T, w.seed, samples=samples)


def pick(gpu, w, samples):
    off = frame_offsets(w)
    idx = off[samples[0]] + samples[1]
    return {k: v[idx] for k, v in gpu.items()}
