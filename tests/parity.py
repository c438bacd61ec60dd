"""Comparison of the CUDA path's dense per-beam output with the oracle.

Tolerances (spec contract): hit triangle, instance and valid mask
bit-exact outside the counted exemptions; range rel 1e-5; intensity rel 1e-4
with an absolute floor of 1e-7 * gain for returns near zero intensity; normal
abs 1e-5.  Exempted beams (oracle flags) are counted, never silently passed.
"""
import numpy as np

RANGE_RTOL = 1e-5
INTENSITY_RTOL = 1e-4
INTENSITY_FLOOR = 1e-7
NORMAL_ATOL = 1e-5

EXEMPT_DISCRETE = 1 | 2 | 4   # edge band, depth tie, cut-off margin
FLAG_SUBTIE = 8
FLAG_GRAZING = 16
NO_HIT = 0xFFFFFFFF


def to_numpy(beams):
    out = {}
    for k, v in beams.items():
        a = v.detach().cpu().numpy()
        if k in ("tri", "inst"):
            a = a.view(np.uint32)
        if k == "mat":
            a = a.view(np.uint16)
        out[k] = a
    return out


def gather(gpu, offsets, sample_frame, sample_beam):
    idx = offsets[sample_frame] + sample_beam
    return {k: v[idx] for k, v in gpu.items()}


def compare(gpu, ref, gain=1.0, label=""):
    """Returns a report dict; raises AssertionError on a mismatch outside the
    exemptions."""
    flags = ref["flags"].astype(np.int64)
    n = flags.size
    subray = ref["sub_I"].shape[1] > 1 and np.any(ref["sub_valid"][:, 1:])
    exempt = (flags & EXEMPT_DISCRETE) != 0
    if subray:
        exempt |= (flags & FLAG_SUBTIE) != 0
    ok = ~exempt
    rep = {"label": label, "beams": int(n), "exempt": int(exempt.sum()),
           "edge": int(((flags & 1) != 0).sum()), "tie": int(((flags & 2) != 0).sum()),
           "cutoff": int(((flags & 4) != 0).sum()), "subtie": int(((flags & 8) != 0).sum()),
           "grazing": int(((flags & 16) != 0).sum())}
    bad_tri = ok & (gpu["tri"] != ref["tri"])
    assert not bad_tri.any(), f"{label}: hit triangle differs on {int(bad_tri.sum())} beams, e.g. " \
                              f"{np.flatnonzero(bad_tri)[:5]}"
    bad_valid = ok & (gpu["valid"].astype(bool) != ref["valid"].astype(bool))
    assert not bad_valid.any(), f"{label}: valid mask differs on {int(bad_valid.sum())} beams, e.g. " \
                                f"{np.flatnonzero(bad_valid)[:5]}"
    h = ok & (ref["tri"] != NO_HIT)
    if "inst" in gpu:
        assert np.array_equal(gpu["inst"][h], ref["inst"][h]), f"{label}: instance differs"
    if "mat" in gpu:
        assert np.array_equal(gpu["mat"][h], ref["mat"][h]), f"{label}: material differs"
    rel = np.abs(gpu["range"][h].astype(np.float64) - ref["range"][h]) / np.abs(ref["range"][h])
    rep["range_max_rel"] = float(rel.max()) if rel.size else 0.0
    assert rep["range_max_rel"] <= RANGE_RTOL, f"{label}: range rel err {rep['range_max_rel']:.3g}"
    dI = np.abs(gpu["intensity"][h].astype(np.float64) - ref["intensity"][h])
    tolI = INTENSITY_RTOL * np.abs(ref["intensity"][h]) + INTENSITY_FLOOR * gain
    rep["intensity_max_rel"] = float((dI / np.maximum(np.abs(ref["intensity"][h]), 1e-30)).max()) if dI.size else 0.0
    bad_I = dI > tolI
    assert not bad_I.any(), f"{label}: intensity differs on {int(bad_I.sum())} beams (max rel " \
                            f"{rep['intensity_max_rel']:.3g})"
    v = h & (ref["valid"] != 0)
    if "normal" in gpu:
        dn = np.abs(gpu["normal"][v].astype(np.float64) - ref["normal"][v]).max() if v.any() else 0.0
        rep["normal_max_abs"] = float(dn)
        assert dn <= NORMAL_ATOL, f"{label}: normal abs err {dn:.3g}"
    rep["hits"] = int(h.sum())
    rep["returns"] = int(v.sum())
    return rep


def compare_subray(gpu, ref, gain=1.0, label=""):
    """Beams with several sub-rays: where the strongest return is unique
    (no SUBTIE flag) compare everything; elsewhere check that the GPU's chosen
    sub-ray is valid in the oracle, that its oracle intensity is the maximum
    within tolerance, and that range and intensity match that sub-ray."""
    rep = compare(gpu, ref, gain, label)
    flags = ref["flags"].astype(np.int64)
    amb = (flags & FLAG_SUBTIE) != 0
    k = gpu["sub"].astype(np.int64)
    rows = np.flatnonzero(amb & (gpu["valid"] != 0))
    n_checked = 0
    for r in rows:
        sub_flags = ref["sub_flags"][r]
        if sub_flags[k[r]] & EXEMPT_DISCRETE:
            continue
        assert ref["sub_valid"][r, k[r]], f"{label}: beam {r} picks a sub-ray the oracle drops"
        Imax = ref["sub_I"][r][ref["sub_valid"][r] != 0].max()
        Ik = ref["sub_I"][r, k[r]]
        assert Imax - Ik <= INTENSITY_RTOL * Imax + INTENSITY_FLOOR * gain, f"{label}: beam {r} not strongest"
        assert abs(gpu["range"][r] - ref["sub_range"][r, k[r]]) <= RANGE_RTOL * ref["sub_range"][r, k[r]]
        assert abs(gpu["intensity"][r] - Ik) <= INTENSITY_RTOL * abs(Ik) + INTENSITY_FLOOR * gain
        n_checked += 1
    rep["subray_ambiguous_checked"] = n_checked
    return rep
