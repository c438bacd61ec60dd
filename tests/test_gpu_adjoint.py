"""Parity of the adjoint (hits and masks frozen) with the oracle's FP64
adjoint, and central finite differences of the GPU loss.

Targets are computed by the oracle (hidden material parameters) and passed to
both sides; beams the oracle flags as ambiguous in either forward pass are
left out of the mask so both sides sum over the same beams."""
import numpy as np
import pytest

import oracle
import synth
from bench import build_cfg1  # the benchmark's hierarchy of the 1M-triangle scene
from gpu_util import frame_offsets, oracle_cast, stratified_sample

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NORM_RTOL = 1e-5


def close_grad(got, ref, label):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(np.linalg.norm(ref), 1e-30)
    rel = np.linalg.norm(got - ref) / scale
    ent = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30)
    assert rel <= NORM_RTOL, f"{label}: norm-relative error {rel:.3g}"
    assert ent <= NORM_RTOL, f"{label}: per-entry error {ent:.3g} of max|g|"
    return rel


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


def _gpu_tape(L, w, scene=None, fields=("valid", "intensity", "mat", "theta_deg", "rf")):
    if scene is None:
        scene = L.build_scene(w.scene.verts, w.scene.tris, w.scene.mat, w.scene.inst)
    for s, spec in enumerate(w.sensors):
        L.set_sensor(s, spec)
    params = torch.tensor(w.params, device=L.device)
    table = L.build_tables(params)
    L.set_materials(table)
    n = L.total_beams(w.frames)
    tape = L.alloc_beams(n, fields)
    L.cast_into(scene, w.frames, w.seed, tape)
    assert L.sync_status() == 0
    return scene, params, table, tape, n


def _targets(w, fwd, tgt, n, idx=None):
    """Oracle targets as FP32 device arrays; mask = target valid, both oracle
    passes unflagged."""
    ok = ((fwd.flags & 7) == 0) & ((tgt.flags & 7) == 0) & (tgt.valid != 0)
    tI = np.zeros(n, np.float32)
    tv = np.zeros(n, np.uint8)
    sel = np.arange(n) if idx is None else idx
    tI[sel] = tgt.intensity.astype(np.float32)
    tv[sel] = ok.astype(np.uint8)
    return tI, tv


def _gpu_backward_mse(L, tape, table, gain, tI, tv):
    dev = L.device
    loss = torch.zeros(1, device=dev)
    gT = torch.zeros_like(table)
    gg = torch.zeros(1, device=dev)
    L.cast_backward_mse(tape, gain, torch.tensor(tI, device=dev), torch.tensor(tv, device=dev), loss, gT, gg)
    assert L.sync_status() == 0
    return loss.item(), gT.cpu().numpy(), gg.item()


def test_adjoint_small_terrain_every_beam(L):
    w = synth.small_terrain(seed=31, n_frames=3, n_az=256)
    scene, params, table, tape, n = _gpu_tape(L, w)
    fwd = oracle_cast(w)
    tgt = oracle_cast(w, table=oracle.build_tables(w.hidden_params))
    tI, tv = _targets(w, fwd, tgt, n)
    loss, gT, gg = _gpu_backward_mse(L, tape, table, 1.0, tI, tv)
    # the oracle sums over the same beams: its own tape, the same targets and mask
    L_ref, gT_ref, gg_ref, N = oracle.cast_backward(fwd.valid, fwd.mat, fwd.theta_deg, fwd.rf,
                                                    oracle.build_tables(w.params), 1.0, tI.astype(np.float64), tv)
    assert N > 1000
    assert loss == pytest.approx(L_ref, rel=NORM_RTOL)
    close_grad(gT, gT_ref, "dL/dT")
    assert gg == pytest.approx(gg_ref, rel=NORM_RTOL)
    gp = L.build_tables_backward(params, torch.tensor(gT, device=L.device)).cpu().numpy()
    gp_ref = oracle.build_tables_backward(w.params, gT_ref)
    close_grad(gp, gp_ref, "dL/d(a,s,w)")


def test_autograd_path_matches_fused_mse(L):
    """LidarCast (torch autograd, generic dL/dI) against the fused-MSE kernel."""
    from paper_2208_10295_gb300 import LidarCast
    w = synth.small_terrain(seed=32, n_frames=2, n_az=256)
    scene, params, table, tape, n = _gpu_tape(L, w)
    fwd = oracle_cast(w)
    tgt = oracle_cast(w, table=oracle.build_tables(w.hidden_params))
    tI, tv = _targets(w, fwd, tgt, n)
    p = params.clone().requires_grad_(True)
    g = torch.tensor(1.0, device=L.device, requires_grad=True)
    I, valid = LidarCast.apply(p, g, L, scene, w.frames, w.seed, 0)
    mask = (valid != 0) & torch.tensor(tv != 0, device=L.device)
    res = (I - torch.tensor(tI, device=L.device))[mask]
    loss = (res * res).sum() / mask.sum()
    loss.backward()
    L.set_materials(table)
    l2, gT, gg = _gpu_backward_mse(L, tape, table, 1.0, tI, tv)
    gp_fused = L.build_tables_backward(params, torch.tensor(gT, device=L.device)).cpu().numpy()
    assert loss.item() == pytest.approx(l2, rel=1e-5)
    close_grad(p.grad.cpu().numpy(), gp_fused, "autograd dL/d(a,s,w)")
    assert g.grad.item() == pytest.approx(gg, rel=1e-5)


def test_adjoint_cfg3_sampled(L):
    """Full 16-frame workload on the GPU; the mask keeps a seeded sample of
    beams that the oracle computes one by one."""
    w = synth.cfg3()
    scene, params, table, tape, n = _gpu_tape(L, w, scene=build_cfg1(L, w))
    samples = stratified_sample(w, 1024, seed=3)
    fwd = oracle_cast(w, samples)
    tgt = oracle_cast(w, samples, table=oracle.build_tables(w.hidden_params))
    idx = frame_offsets(w)[samples[0]] + samples[1]
    tI, tv = _targets(w, fwd, tgt, n, idx)
    loss, gT, gg = _gpu_backward_mse(L, tape, table, 1.0, tI, tv)
    L_ref, gT_ref, gg_ref, N = oracle.cast_backward(fwd.valid, fwd.mat, fwd.theta_deg, fwd.rf,
                                                    oracle.build_tables(w.params), 1.0,
                                                    tI[idx].astype(np.float64), tv[idx])
    assert N > 200
    assert loss == pytest.approx(L_ref, rel=NORM_RTOL)
    close_grad(gT, gT_ref, "cfg3 dL/dT")
    assert gg == pytest.approx(gg_ref, rel=NORM_RTOL)
    _check_params_grad(L, params, gT, w.params, gT_ref, "cfg3")


def _check_params_grad(L, params, gT, params_np, gT_ref, label):
    """dL/d(a, s, w) through the table builder's chain rule: the GPU's builder
    backward applied to the GPU's dL/dT against the oracle's FP64 builder
    backward applied to the oracle's dL/dT, for the three columns together
    and for the specular width on its own (its gradient is an order of
    magnitude below the albedo's, so the joint check alone would not see it)."""
    gp = L.build_tables_backward(params, torch.tensor(gT, device=L.device)).cpu().numpy()
    gp_ref = oracle.build_tables_backward(params_np, gT_ref)
    close_grad(gp, gp_ref, f"{label} dL/d(a,s,w)")
    close_grad(gp[:, 2], gp_ref[:, 2], f"{label} dL/dw (specular width)")


def test_cfg3_finite_differences_full_size(L):
    """All 4.2M beams: the frozen-hit loss is quadratic in T and g, so central
    differences of the GPU loss match its gradient (rel 1e-3)."""
    w = synth.cfg3()
    scene, params, table, tape, n = _gpu_tape(L, w, scene=build_cfg1(L, w))
    dev = L.device
    Th = L.build_tables(torch.tensor(w.hidden_params, device=dev))
    L.set_materials(Th)
    tgt = L.alloc_beams(n, ("valid", "intensity", "mat", "theta_deg", "rf"))
    L.cast_into(scene, w.frames, w.seed, tgt)
    L.set_materials(table)
    tI = tgt["intensity"]
    tv = tgt["valid"]
    loss0, gT, gg = _gpu_backward_mse(L, tape, table, 1.0, tI.cpu().numpy(), tv.cpu().numpy())
    assert loss0 > 0
    rng = np.random.default_rng(0)
    # entries carrying at least 1% of the largest gradient; the loss is exactly
    # quadratic in T, so a large step h adds no truncation error and keeps the
    # FP32 loss difference well above its rounding
    used = np.argwhere(np.abs(gT) > 1e-2 * np.abs(gT).max())
    for m, k in used[rng.choice(len(used), 6, replace=False)]:
        h = 0.5
        vals = []
        for sgn in (1, -1):
            Tp = table.clone()
            Tp[m, k] += sgn * h
            L.set_materials(Tp)
            lval, _, _ = _gpu_backward_mse(L, tape, Tp, 1.0, tI.cpu().numpy(), tv.cpu().numpy())
            vals.append(lval)
        L.set_materials(table)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert gT[m, k] == pytest.approx(fd, rel=1e-3, abs=1e-6 * np.abs(gT).max()), (m, k)
    vals = []
    for sgn in (1, -1):
        lval, _, _ = _gpu_backward_mse(L, tape, table, 1.0 + sgn * 0.25, tI.cpu().numpy(), tv.cpu().numpy())
        vals.append(lval)
    assert gg == pytest.approx((vals[0] - vals[1]) / 0.5, rel=1e-3)


def test_adjoint_deterministic(L):
    w = synth.small_terrain(seed=33, n_frames=2, n_az=256)
    scene, params, table, tape, n = _gpu_tape(L, w)
    rng = np.random.default_rng(1)
    tI = rng.uniform(0, 0.5, n).astype(np.float32)
    tv = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    a = _gpu_backward_mse(L, tape, table, 1.0, tI, tv)
    b = _gpu_backward_mse(L, tape, table, 1.0, tI, tv)
    assert a[0] == b[0] and a[2] == b[2]
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


def test_adjoint_unaligned_tape_matches_aligned(L):
    """Tape arrays that start one element past an aligned address take the
    scalar-load path; over the same beams it gives the same gradients bit for
    bit (fixed-point sums) as the vector-load path on an aligned copy, and the
    loss to rounding."""
    w = synth.small_terrain(seed=34, n_frames=2, n_az=256)
    scene, params, table, tape, n = _gpu_tape(L, w)
    rng = np.random.default_rng(2)
    tI = torch.tensor(rng.uniform(0, 0.5, n).astype(np.float32), device=L.device)
    tv = torch.tensor((rng.uniform(size=n) < 0.7).astype(np.uint8), device=L.device)
    off = {k: v[1:] for k, v in tape.items()}                       # unaligned views
    same = {k: v[1:].clone() for k, v in tape.items()}              # aligned copies of the same beams
    outs = []
    for tp, ti, tvv in ((off, tI[1:], tv[1:]), (same, tI[1:].clone(), tv[1:].clone())):
        loss = torch.zeros(1, device=L.device)
        gT = torch.zeros_like(table)
        gg = torch.zeros(1, device=L.device)
        L.cast_backward_mse(tp, 1.0, ti, tvv, loss, gT, gg)
        assert L.sync_status() == 0
        outs.append((loss.item(), gT.cpu().numpy(), gg.item()))
    (la, ga, gga), (lb, gb, ggb) = outs
    assert np.array_equal(ga.view(np.uint32), gb.view(np.uint32)) and gga == ggb
    assert la == pytest.approx(lb, rel=1e-12)


def test_adjoint_city_sampled(L):
    """cfg4 forward + adjoint: the 10.7M-triangle city, all 32 frames with 7
    sub-rays per beam on the GPU (tape of each beam's strongest sub-ray); the
    mask keeps a seeded sample of beams that the oracle recomputes, where both
    pick the same sub-ray and nothing is exempt; targets from the hidden
    64-material table.  Loss and gradients against the oracle's adjoint."""
    from bench import build_city  # the benchmark's hierarchy of the city
    w = synth.cfg4()
    scene, params, table, tape, n = _gpu_tape(L, w, scene=build_city(L, w),
                                              fields=("valid", "intensity", "mat", "theta_deg", "rf", "sub"))
    samples = stratified_sample(w, 256, seed=6)
    fwd = oracle_cast(w, samples)
    tgt = oracle_cast(w, samples, table=oracle.build_tables(w.hidden_params))
    idx = frame_offsets(w)[samples[0]] + samples[1]
    gsub = tape["sub"].cpu().numpy()[idx].astype(np.int64)
    r = np.arange(idx.size)
    ok = (((fwd.flags & 7) == 0) & ((tgt.flags & 7) == 0) & (tgt.valid != 0) & (gsub == fwd.sub) &
          ((fwd.sub_flags[r, np.clip(fwd.sub, 0, None)] & 7) == 0))
    tI = np.zeros(n, np.float32)
    tv = np.zeros(n, np.uint8)
    tI[idx] = tgt.intensity.astype(np.float32)
    tv[idx] = ok.astype(np.uint8)
    loss, gT, gg = _gpu_backward_mse(L, tape, table, 1.0, tI, tv)
    L_ref, gT_ref, gg_ref, N = oracle.cast_backward(fwd.valid, fwd.mat, fwd.theta_deg, fwd.rf,
                                                    oracle.build_tables(w.params), 1.0,
                                                    tI[idx].astype(np.float64), tv[idx])
    assert N > 30
    assert loss == pytest.approx(L_ref, rel=NORM_RTOL)
    close_grad(gT, gT_ref, "city dL/dT")
    assert gg == pytest.approx(gg_ref, rel=NORM_RTOL)
    _check_params_grad(L, params, gT, w.params, gT_ref, "city")


# ----------------------------------------------------------------- synthetic tapes
# The adjoint alone on tapes drawn directly (no cast), against the oracle's FP64
# adjoint on the same FP32 inputs: sizes that leave a partial last chunk, enough
# chunks per SM that every block streams several through its copy stages, a
# target scale that keeps growing inside each block (its fixed-point sums are
# rescaled on the way), material ids past the table, a table too large for
# shared memory (the separate passes), and the empty and one-beam tapes.

def _synthetic(L, n, M, seed):
    t = synth.adjoint_tape(n, M, seed)
    dev = L.device
    params = torch.tensor(t["params"], device=dev)
    table = L.build_tables(params)
    L.set_materials(table)
    tape = {k: torch.tensor(t[k], device=dev) for k in ("valid", "mat", "theta_deg", "rf")}
    return t, params, table, tape, torch.tensor(t["target_I"], device=dev), torch.tensor(t["target_valid"], device=dev)


def _mse(L, tape, table, tI, tv, gain):
    loss = torch.zeros(1, device=L.device)
    gT = torch.zeros_like(table)
    gg = torch.zeros(1, device=L.device)
    L.cast_backward_mse(tape, gain, tI, tv, loss, gT, gg)
    st = L.sync_status()
    assert st == 0, st
    return loss.item(), gT.cpu().numpy(), gg.item()


@pytest.mark.parametrize("n,M", [(2_500_001, 32), (4_194_304, 64), (3000, 64), (2048, 4), (1, 8), (0, 8),
                                 (200_003, 200)])
def test_adjoint_synthetic_tape_vs_oracle(L, n, M):
    t, params, table, tape, tI, tv = _synthetic(L, n, M, seed=7000 + M + n % 97)
    gain = 1.25
    loss, gT, gg = _mse(L, tape, table, tI, tv, gain)
    T = table.cpu().numpy().astype(np.float64)
    L_ref, gT_ref, gg_ref, N = oracle.cast_backward(t["valid"], t["mat"], t["theta_deg"], t["rf"], T, gain,
                                                    t["target_I"].astype(np.float64), t["target_valid"])
    if N == 0:
        assert loss == 0.0 and gg == 0.0 and not gT.any()
        return
    assert loss == pytest.approx(L_ref, rel=NORM_RTOL)
    close_grad(gT, gT_ref, f"synthetic n={n} M={M} dL/dT")
    assert gg == pytest.approx(gg_ref, rel=NORM_RTOL)


@pytest.mark.parametrize("M", [32, 200])
def test_adjoint_count_and_split_tape_combined(L, M):
    """`n_used` is the number of beams valid in both tape and targets (the one
    -pass kernel for 32 materials, the separate passes for 200), and a tape
    split in three uneven parts, each part's adjoint combined by its count
    (`combine_mse`, the arithmetic the ranks of a sharded fit all-reduce),
    gives the whole tape's loss and gradients."""
    from paper_2208_10295_gb300.torch_api import combine_mse
    n = 1_000_003
    t, params, table, tape, tI, tv = _synthetic(L, n, M, seed=7300 + M)
    dev = L.device

    def run(lo, hi):
        loss = torch.zeros(1, device=dev)
        gT = torch.zeros_like(table)
        gg = torch.zeros(1, device=dev)
        cnt = torch.full((1,), -1, dtype=torch.int64, device=dev)
        L.cast_backward_mse({k: v[lo:hi] for k, v in tape.items()}, 1.25, tI[lo:hi], tv[lo:hi], loss, gT, gg,
                            n_used=cnt)
        assert L.sync_status() == 0
        return loss, gT, gg, cnt

    whole = run(0, n)
    expect = int(((t["valid"] != 0) & (t["target_valid"] != 0)).sum())
    assert int(whole[3].item()) == expect
    cuts = [0, 123_457, 700_001, n]
    parts = [run(a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert sum(int(p[3].item()) for p in parts) == expect
    loss = torch.zeros(1, device=dev)
    gT = torch.zeros_like(table)
    gg = torch.zeros(1, device=dev)
    total = combine_mse(parts, loss, gT, gg)
    assert int(total.item()) == expect
    assert loss.item() == pytest.approx(whole[0].item(), rel=1e-6)
    close_grad(gT.cpu().numpy(), whole[1].cpu().numpy(), f"split tape M={M} dL/dT")
    assert gg.item() == pytest.approx(whole[2].item(), rel=1e-6)


def test_adjoint_synthetic_unaligned_and_repeat_bit_identical(L):
    """Tape views one element past an aligned address (the threads load the
    tape; no copy engine) give the gradients of aligned copies of the same
    beams (copied by the copy engine) bit for bit, and a repeated call gives
    the same bits again."""
    n = 1_500_007
    t, params, table, tape, tI, tv = _synthetic(L, n, 32, seed=7100)
    off = {k: v[1:] for k, v in tape.items()}
    same = {k: v[1:].clone() for k, v in tape.items()}
    a = _mse(L, off, table, tI[1:], tv[1:], 1.0)
    b = _mse(L, same, table, tI[1:].clone(), tv[1:].clone(), 1.0)
    c = _mse(L, same, table, tI[1:].clone(), tv[1:].clone(), 1.0)
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32)) and a[2] == b[2]
    assert np.array_equal(b[1].view(np.uint32), c[1].view(np.uint32)) and b[2] == c[2] and b[0] == c[0]
    assert a[0] == pytest.approx(b[0], rel=1e-12)


def test_adjoint_wait_runs_out_and_recovers(L):
    """The adjoint's bounded waits (copy stages, grid-wide wait) made to run
    out with a 0 ns limit: the call reports LIDAR_ETIMEOUT through the status
    word, nothing hangs, and with the default limit back the next call gives
    the reference result bit for bit."""
    from paper_2208_10295_gb300 import capi
    t, params, table, tape, tI, tv = _synthetic(L, 2_000_000, 32, seed=7200)
    ref = _mse(L, tape, table, tI, tv, 1.0)
    limit0 = L.wait_limit()
    try:
        L.set_wait_limit(0)
        loss = torch.zeros(1, device=L.device)
        gT = torch.zeros_like(table)
        gg = torch.zeros(1, device=L.device)
        L.cast_backward_mse(tape, 1.0, tI, tv, loss, gT, gg)
        assert L.sync_status() == capi.LIDAR_ETIMEOUT
    finally:
        L.set_wait_limit(limit0)
    again = _mse(L, tape, table, tI, tv, 1.0)
    assert again[0] == ref[0] and again[2] == ref[2]
    assert np.array_equal(again[1].view(np.uint32), ref[1].view(np.uint32))
