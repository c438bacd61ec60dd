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


def _hand_case():
    """Five beams with dyadic inputs, worked out by hand (every value below is
    exact in FP64).  M = 2 material rows; gain g = 2.
      beam 0: material 0, theta 10 (integer: R = T[0][10] = 0.5), rf 0.5,
              I = 2 * 0.5 * 0.5 = 0.5, target 0.25 -> residual +0.25
      beam 1: material 1, theta 30.25 (i 30, f 0.25:
              R = 0.75 T[1][30] + 0.25 T[1][31] = 0.75 * 0.25 + 0.25 * 0.75 = 0.375),
              rf 1, I = 0.75, target 1 -> residual -0.25
      beam 2: valid = 0 (its residual would be large): not in the mask
      beam 3: target_valid = 0: not in the mask
      beam 4: material 5 >= M uses the last row (1); theta 90 (i 89, f 1:
              R = T[1][90] = 0.125), rf 2, I = 2 * 2 * 0.125 = 0.5, target 0
              -> residual +0.5
    N = 3 beams in both masks; L = (0.0625 + 0.0625 + 0.25) / 3 = 0.125.
    dL/dI_b = 2 r_b / N = +1/6, -1/6, +1/3 for beams 0, 1, 4:
      dT[0][10] = g rf (1 - f) dL/dI = 2 * 0.5 * 1 * 1/6 = 1/6   (dT[0][11] gets f = 0)
      dT[1][30] = 2 * 1 * 0.75 * (-1/6) = -1/4,  dT[1][31] = 2 * 1 * 0.25 * (-1/6) = -1/12
      dT[1][90] = 2 * 2 * 1 * 1/3 = 4/3          (dT[1][89] gets 1 - f = 0)
      dL/dg = sum rf R dL/dI = 0.25/6 - 0.375/6 + 0.25/3 = 1/24 - 1/16 + 1/12 = 1/16."""
    T = np.zeros((2, 91))
    T[0, 10] = 0.5
    T[0, 11] = 0.875          # reached only with weight f = 0
    T[1, 30] = 0.25
    T[1, 31] = 0.75
    T[1, 89] = 0.625          # reached only with weight 1 - f = 0
    T[1, 90] = 0.125
    T[0, 40] = 1.0            # beams 2 and 3 would read here
    valid = np.array([1, 1, 0, 1, 1], np.uint8)
    target_valid = np.array([1, 1, 1, 0, 1], np.uint8)
    mat = np.array([0, 1, 0, 0, 5], np.uint16)
    theta = np.array([10.0, 30.25, 40.0, 40.0, 90.0])
    rf = np.array([0.5, 1.0, 1.0, 1.0, 2.0])
    target = np.array([0.25, 1.0, -7.0, -7.0, 0.0])
    return (valid, mat, theta, rf), T, 2.0, target, target_valid


def test_loss_hand_computed_case(oracle_lib):
    """The loss's value itself (not only its gradient relative to it): the
    mask (both validity flags), the normalisation by N, the interpolation,
    the material clamp and the theta = 90 end of the table, on a case worked
    out by hand."""
    args, T, g, target, tv = _hand_case()
    assert oracle_lib.loss(*args, T, g, target, tv) == 0.125
    L, gT, gg, N = oracle_lib.cast_backward(*args, T, g, target, tv)
    assert N == 3 and L == 0.125
    want = np.zeros_like(T)
    want[0, 10] = 1 / 6
    want[1, 30] = -0.25
    want[1, 31] = -1 / 12
    want[1, 90] = 4 / 3
    assert np.allclose(gT, want, rtol=1e-15, atol=0.0)
    assert gg == pytest.approx(1 / 16, rel=1e-15)
    # flipping a beam's forward flag moves it into or out of the mask exactly
    # when its target flag is set (beam 3's never is)
    for b in range(5):
        v2 = args[0].copy()
        v2[b] ^= 1
        changed = oracle_lib.loss(v2, *args[1:], T, g, target, tv) != 0.125
        assert changed == bool(tv[b]), b
