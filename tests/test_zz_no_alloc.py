"""The allocation-free adjoint entry point, for callers that must not allocate
device memory (hard real-time loops that cannot take cudaMalloc's implicit
synchronisation, hosts whose memory pool owns the device).  Its scratch is a
fixed array inside the library.

Checked through the C ABI against lidar_cast_backward_mse on the same tape and
targets, on two calls in a row (the shared scratch must be cleared between
calls).  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-5   # norm-relative tolerance the adjoint tests use


def _close(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) <= GRAD_RTOL * max(np.linalg.norm(b), 1e-30)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_10295_gb300 import Lidar
    L = Lidar(0)
    w = synth.small_terrain(seed=21, n_frames=2, n_az=256)
    scene = L.build_scene(w.scene.verts, w.scene.tris, w.scene.mat, w.scene.inst)
    L.set_sensor(0, w.sensors[0])
    dev = L.device
    table_h = L.build_tables(torch.tensor(w.hidden_params, device=dev))
    L.set_materials(table_h)
    n = L.total_beams(w.frames)
    tgt = L.alloc_beams(n, ("valid", "intensity", "mat", "theta_deg", "rf"))
    L.cast_into(scene, w.frames, w.seed, tgt)
    table = L.build_tables(torch.tensor(w.params, device=dev))
    L.set_materials(table)
    tape = L.alloc_beams(n, ("valid", "intensity", "mat", "theta_deg", "rf"))
    L.cast_into(scene, w.frames, w.seed, tape)
    assert L.sync_status() == 0
    yield L, tape, tgt, table, n
    L.close()


def _reference(L, tape, tgt, table):
    loss = torch.zeros(1, device=L.device)
    gT = torch.zeros_like(table)
    gg = torch.zeros(1, device=L.device)
    L.cast_backward_mse(tape, 1.0, tgt["intensity"], tgt["valid"], loss, gT, gg)
    torch.cuda.synchronize()
    return loss.item(), gT.cpu().numpy(), gg.item()


def _outputs(L, table):
    return torch.zeros(1, device=L.device), torch.zeros_like(table), torch.zeros(1, device=L.device)


def _noalloc(L, tape, tgt, table, n, outs):
    from paper_2208_10295_gb300 import capi
    loss, gT, gg = outs
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = capi.lidar_cast_backward_mse_noalloc(
        ctypes.c_void_p(L.stream.cuda_stream), n, p(tape["valid"]), p(tape["mat"]), p(tape["theta_deg"]),
        p(tape["rf"]), p(table), table.shape[0], 1.0, p(tgt["intensity"]), p(tgt["valid"]), p(loss), p(gT), p(gg))
    assert st == capi.LIDAR_OK, capi.last_error()
    torch.cuda.synchronize()
    return loss.item(), gT.cpu().numpy(), gg.item()


def test_noalloc_backward_matches_allocating_entry_point(setup):
    L, tape, tgt, table, n = setup
    ref = _reference(L, tape, tgt, table)
    assert np.abs(ref[1]).sum() > 0
    # first call (also performs the once-per-device address lookup)
    first = _noalloc(L, tape, tgt, table, n, _outputs(L, table))
    # second call in a row: must not see the first call's accumulators, and
    # must leave the device's free memory unchanged
    outs = _outputs(L, table)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    second = _noalloc(L, tape, tgt, table, n, outs)
    free1, _ = torch.cuda.mem_get_info()
    assert free0 == free1
    for got in (first, second):
        assert got[0] == pytest.approx(ref[0], rel=GRAD_RTOL)
        assert _close(got[1], ref[1])
        assert got[2] == pytest.approx(ref[2], rel=GRAD_RTOL, abs=1e-12)


def test_noalloc_rejects_too_many_materials(setup):
    from paper_2208_10295_gb300 import capi
    L, tape, tgt, table, n = setup
    big = torch.zeros((65, 91), device=L.device)
    st = capi.lidar_cast_backward_mse_noalloc(None, 0, None, None, None, None, ctypes.c_void_p(big.data_ptr()), 65,
                                              1.0, None, None, None, None, None)
    assert st == capi.LIDAR_EINVAL
    assert "exceed" in capi.last_error()
