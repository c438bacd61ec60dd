"""Pins of the oracle's building blocks against definitions outside the oracle:
Python's libm, exact-rational replay of FP32 operations, numpy's Philox,
distributional properties, and finite differences."""
import math

import numpy as np
import pytest

from exact import f32_add, f32_div, f32_fma, f32_mul, f32_sqrt, f32_sub


def test_beam_dirs_follow_spherical_definition(oracle_lib):
    rng = np.random.default_rng(1)
    az = rng.uniform(0, 2 * np.pi, 500)
    el = rng.uniform(-np.pi / 2, np.pi / 2, 500)
    got = oracle_lib.beam_dirs(az, el)
    for k in range(500):
        ce = math.cos(el[k])
        want = np.array([ce * math.cos(az[k]), ce * math.sin(az[k]), math.sin(el[k])], dtype=np.float32)
        assert np.array_equal(got[k], want)
    # the azimuth-zero beam has an exact zero y component
    z = oracle_lib.beam_dirs([0.0], [0.1])
    assert z[0, 1] == 0.0


def test_world_ray_is_exact_fp32_fma_replay(oracle_lib):
    rng = np.random.default_rng(2)
    for _ in range(200):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                      [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                      [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        pose = np.concatenate([R, rng.uniform(-300, 300, (3, 1))], 1).reshape(12).astype(np.float32)
        d = rng.normal(size=3).astype(np.float32)
        o, dw = oracle_lib.world_ray(pose, d)
        P = pose.reshape(3, 4)
        for r in range(3):
            p0 = f32_mul(P[r, 0], d[0])
            acc = f32_fma(P[r, 1], d[1], p0)
            want = f32_fma(P[r, 2], d[2], acc)
            assert dw[r] == want
            assert o[r] == P[r, 3]


def _subray_replay(d, alpha, beta):
    d = [np.float32(x) for x in d]
    n2 = f32_add(f32_mul(d[1], d[1]), f32_mul(d[0], d[0]))
    if f32_sqrt(n2) >= np.float32(1e-3):
        c = [d[1], np.float32(-d[0]), np.float32(0.0)]
    else:
        c = [np.float32(0.0), d[2], np.float32(-d[1])]
    cc = f32_add(f32_add(f32_mul(c[0], c[0]), f32_mul(c[1], c[1])), f32_mul(c[2], c[2]))
    s = f32_sqrt(cc)
    u = [f32_div(ci, s) for ci in c]
    v = [f32_sub(f32_mul(d[1], u[2]), f32_mul(d[2], u[1])),
         f32_sub(f32_mul(d[2], u[0]), f32_mul(d[0], u[2])),
         f32_sub(f32_mul(d[0], u[1]), f32_mul(d[1], u[0]))]
    w = [f32_add(f32_add(d[i], f32_mul(alpha, u[i])), f32_mul(beta, v[i])) for i in range(3)]
    ww = f32_add(f32_add(f32_mul(w[0], w[0]), f32_mul(w[1], w[1])), f32_mul(w[2], w[2]))
    sw = f32_sqrt(ww)
    return np.array([f32_div(wi, sw) for wi in w], dtype=np.float32)


def test_subray_offsets_and_dirs(oracle_lib):
    a, b = oracle_lib.subray_offsets(1e-4, 7)
    assert a[0] == 0 and b[0] == 0
    r = math.tan(0.5 * float(np.float32(1e-4)))
    for k in range(1, 7):
        ang = 2 * math.pi * (k - 1) / 6
        assert a[k] == np.float32(r * math.cos(ang))
        assert b[k] == np.float32(r * math.sin(ang))
    rng = np.random.default_rng(3)
    dirs = rng.normal(size=(60, 3)).astype(np.float32)
    dirs[0] = [1e-5, 2e-5, 1.0]        # near the pole: takes the x-hat branch
    dirs[1] = [0.0, 0.0, -1.0]
    for d in dirs:
        for k in range(7):
            got = oracle_lib.subray_dir(d, a[k], b[k], k)
            if k == 0:
                assert np.array_equal(got, d)
            else:
                assert np.array_equal(got, _subray_replay(d, a[k], b[k]))
    # the perturbed rays sit at the stated half-angle from the beam (beam
    # directions are unit vectors rounded to float32)
    d = (np.array([0.3, -0.4, 0.5]) / np.linalg.norm([0.3, -0.4, 0.5])).astype(np.float32)
    dn = d.astype(np.float64) / np.linalg.norm(d.astype(np.float64))
    for k in range(1, 7):
        s = oracle_lib.subray_dir(d, a[k], b[k], k).astype(np.float64)
        ang = math.acos(min(1.0, float(s @ dn) / np.linalg.norm(s)))
        assert abs(ang - 0.5e-4) < 2e-6


def _numpy_philox_block(ctr, key):
    """numpy.random.Philox returns the block for counter c+1: step back by one."""
    c = [int(x) for x in ctr]
    for i in range(4):  # 256-bit decrement with borrow (wraps at zero)
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = 2 ** 64 - 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return bg.random_raw(4)


def test_philox_matches_numpy(oracle_lib):
    rng = np.random.default_rng(4)
    cases = [([0, 0, 0, 0], [0, 0]), ([1, 0, 0, 0], [5, 0]), ([7, 0, 1, 0], [2002, 0])]
    for _ in range(40):
        cases.append((list(rng.integers(0, 2 ** 63, 4, dtype=np.uint64)),
                      list(rng.integers(0, 2 ** 63, 2, dtype=np.uint64))))
    for ctr, key in cases:
        got = oracle_lib.philox4x64_10(ctr, key)
        want = _numpy_philox_block(ctr, key)
        assert np.array_equal(got, want), (ctr, key)


def test_normal_noise_distribution(oracle_lib):
    scipy_stats = pytest.importorskip("scipy.stats")
    z = np.array([oracle_lib.normal(2000, b, 3, 1, 0) for b in range(60000)])
    assert abs(z.mean()) < 0.015
    assert abs(z.var() - 1.0) < 0.02
    assert abs(scipy_stats.kurtosis(z, fisher=False) - 3.0) < 0.08
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-3
    # Box-Muller output is bounded by sqrt(2 * 53 ln 2) for 53-bit uniforms
    assert np.abs(z).max() < math.sqrt(2 * 53 * math.log(2)) + 1e-9
    # different counters (frame, sensor, sub-ray) give independent draws
    z2 = np.array([oracle_lib.normal(2000, b, 3, 1, 1) for b in range(20000)])
    assert abs(np.corrcoef(z[:20000], z2)[0, 1]) < 0.03


def test_table_builder_closed_forms(oracle_lib):
    params = np.array([[0.5, 0.0, 5.0], [0.25, 0.5, 4.0], [0.8, 0.125, 10.0]], np.float32)
    T = oracle_lib.build_tables(params)
    assert T.shape == (3, 91)
    # Eq. 4 with R(0) = a when the lobe is absent
    assert T[0, 0] == pytest.approx(0.5, abs=1e-15)
    assert T[0, 60] == pytest.approx(0.25, abs=1e-15)
    assert T[0, 90] == pytest.approx(0.0, abs=1e-15)
    # lobe peak at normal incidence, one standard width out it is s * e^{-1/2}
    assert T[1, 0] == pytest.approx(0.75, abs=1e-15)
    assert T[1, 4] - 0.25 * math.cos(math.radians(4)) == pytest.approx(0.5 * math.exp(-0.5), abs=1e-15)
    assert T[2, 10] - float(np.float32(0.8)) * math.cos(math.radians(10)) == pytest.approx(0.125 * math.exp(-0.5), abs=1e-15)


def test_table_builder_backward_matches_central_differences(oracle_lib):
    """Backward of the builder against central differences of the oracle's own
    forward, with perturbations that are exact in float32."""
    rng = np.random.default_rng(5)
    params = np.array([[0.3, 0.2, 3.0], [0.6, 0.1, 7.5]], np.float32)
    G = rng.normal(size=(2, 91))
    got = oracle_lib.build_tables_backward(params, G)
    for m in range(2):
        for j in range(3):
            h = np.float32(2.0 ** -12 * max(1.0, abs(float(params[m, j]))))
            pp = params.copy(); pp[m, j] += h
            pm = params.copy(); pm[m, j] -= h
            fd = float((G * oracle_lib.build_tables(pp)).sum() - (G * oracle_lib.build_tables(pm)).sum())
            fd /= float(pp[m, j]) - float(pm[m, j])
            assert got[m, j] == pytest.approx(fd, rel=2e-5, abs=1e-9)
