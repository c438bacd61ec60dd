"""Pins of the oracle adjoint: central finite differences of the oracle's own
mean-squared intensity loss (hits and masks frozen), through the table
builder for the material parameters."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def tape(oracle_lib):
    w = synth.small_terrain(n_cells=24, half=12.0, n_objects=8, n_frames=2, n_az=96)
    T = oracle_lib.build_tables(w.params)
    Th = oracle_lib.build_tables(w.hidden_params)
    fwd = oracle_lib.cast(w.scene, w.sensors, w.frames, T, w.seed)
    tgt = oracle_lib.cast(w.scene, w.sensors, w.frames, Th, w.seed)
    return w, T, fwd, tgt


def test_adjoint_table_and_gain_exact_central_differences(oracle_lib, tape):
    w, T, fwd, tgt = tape
    g = 1.25
    args = (fwd.valid, fwd.mat, fwd.theta_deg, fwd.rf)
    L, gT, gg, N = oracle_lib.cast_backward(*args, T, g, tgt.intensity, tgt.valid)
    assert N > 500
    assert L == pytest.approx(oracle_lib.loss(*args, T, g, tgt.intensity, tgt.valid), rel=1e-14)
    # the loss is quadratic in T and g: central differences are exact up to rounding
    rng = np.random.default_rng(0)
    used = np.argwhere(np.abs(gT) > 0)
    for (m, k) in used[rng.choice(len(used), 40, replace=False)]:
        h = 1e-3
        Tp = T.copy(); Tp[m, k] += h
        Tm = T.copy(); Tm[m, k] -= h
        fd = (oracle_lib.loss(*args, Tp, g, tgt.intensity, tgt.valid) -
              oracle_lib.loss(*args, Tm, g, tgt.intensity, tgt.valid)) / (2 * h)
        assert gT[m, k] == pytest.approx(fd, rel=1e-7, abs=1e-12)
    # entries no beam touches have zero gradient
    assert np.count_nonzero(gT) < gT.size
    h = 1e-3
    fd = (oracle_lib.loss(*args, T, g + h, tgt.intensity, tgt.valid) -
          oracle_lib.loss(*args, T, g - h, tgt.intensity, tgt.valid)) / (2 * h)
    assert gg == pytest.approx(fd, rel=1e-7)


def test_adjoint_through_builder_matches_fd_in_width(oracle_lib, tape):
    w, _T, fwd, tgt = tape
    g = 1.0
    args = (fwd.valid, fwd.mat, fwd.theta_deg, fwd.rf)
    params = w.params.astype(np.float32)
    T = oracle_lib.build_tables(params)
    _, gT, _, _ = oracle_lib.cast_backward(*args, T, g, tgt.intensity, tgt.valid)
    gp = oracle_lib.build_tables_backward(params, gT)
    for m in range(params.shape[0]):
        for j in range(3):
            hh = np.float32(2.0 ** -10 * max(1.0, abs(float(params[m, j]))))
            pp = params.copy(); pp[m, j] += hh
            pm = params.copy(); pm[m, j] -= hh
            fd = (oracle_lib.loss(*args, oracle_lib.build_tables(pp), g, tgt.intensity, tgt.valid) -
                  oracle_lib.loss(*args, oracle_lib.build_tables(pm), g, tgt.intensity, tgt.valid))
            fd /= float(pp[m, j]) - float(pm[m, j])
            assert gp[m, j] == pytest.approx(fd, rel=1e-3, abs=1e-9), (m, j)


def test_adjoint_empty_mask(oracle_lib, tape):
    _w, T, fwd, tgt = tape
    L, gT, gg, N = oracle_lib.cast_backward(fwd.valid, fwd.mat, fwd.theta_deg, fwd.rf, T, 1.0, tgt.intensity,
                                            np.zeros_like(tgt.valid))
    assert N == 0 and L == 0.0 and gg == 0.0 and not gT.any()
