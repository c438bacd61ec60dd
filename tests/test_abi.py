"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/lidar.h declares; the Python binding covers
them; the oracle and the CUDA path stay independent."""
import ast
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lidar.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:lidar_status|void|const char\*)\s+(lidar_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2208_10295_gb300.build import build
    return build()


def test_library_exports_every_declared_symbol(libpath):
    names = declared_functions()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(lidar_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in names:
        assert getattr(lib, n) is not None


def test_binding_covers_the_header(libpath):
    from paper_2208_10295_gb300 import capi
    names = declared_functions()
    assert sorted(capi.EXPORTED) == names
    capi.load(libpath)
    for n in names:
        assert callable(getattr(capi, n))


def test_last_error_without_gpu(libpath):
    from paper_2208_10295_gb300 import capi
    capi.load(libpath)
    # argument checks run on the host before any device call
    st = capi.lidar_create(0, None, None)
    assert st == capi.LIDAR_EINVAL
    assert "out is NULL" in capi.last_error()
    st = capi.lidar_set_materials(None, None, 0)
    assert st == capi.LIDAR_EINVAL


def _imports(path):
    tree = ast.parse(open(path).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def test_oracle_and_cuda_path_are_independent():
    pkg = os.path.join(ROOT, "paper_2208_10295_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            p = os.path.join(dirpath, f)
            if f.endswith(".py"):
                assert "oracle" not in _imports(p), p
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                assert "lidar_oracle" not in open(p).read(), p
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        p = os.path.join(odir, f)
        if f.endswith(".py"):
            assert "paper_2208_10295_gb300" not in _imports(p), p
        if f.endswith((".c", ".h", ".py")):
            txt = open(p).read()
            assert "lidar.h" not in txt and "csrc" not in txt, p
    # the shared input generators hold no part of the model
    for f in os.listdir(os.path.join(ROOT, "synth")):
        if f.endswith(".py"):
            mods = _imports(os.path.join(ROOT, "synth", f))
            assert "oracle" not in mods and "paper_2208_10295_gb300" not in mods


def test_wait_limit_argument_checks(libpath):
    from paper_2208_10295_gb300 import capi
    capi.load(libpath)
    assert capi.lidar_set_wait_limit(None, 0) == capi.LIDAR_EINVAL
    assert capi.lidar_get_wait_limit(None, None) == capi.LIDAR_EINVAL


def test_autograd_function_rejects_frames_of_other_slots():
    """LidarCast differentiates one sensor slot's gain: frames naming another
    slot are refused before anything reaches the device."""
    import numpy as np
    import torch

    import synth
    from paper_2208_10295_gb300 import LidarCast
    w = synth.small_terrain(seed=1, n_frames=2, n_az=8)
    fr = w.frames.copy()
    fr["sensor"][1] = 3
    p = torch.tensor(np.asarray(w.params, np.float32), requires_grad=True)
    g = torch.tensor(1.0, requires_grad=True)
    with pytest.raises(ValueError, match="slot 0"):
        LidarCast.apply(p, g, None, None, fr, w.seed, 0)


def test_cast_overlap_argument_checks(libpath):
    from paper_2208_10295_gb300 import capi
    capi.load(libpath)
    assert capi.lidar_set_cast_overlap(None, 1) == capi.LIDAR_EINVAL
    assert capi.lidar_get_cast_overlap(None, None) == capi.LIDAR_EINVAL


def test_header_is_plain_c():
    """include/lidar.h is a C header: it compiles as C99 (and as C++17) with
    warnings as errors, so C callers can use the ABI without a C++ compiler."""
    import shutil
    import subprocess
    for cc, args in (("gcc", ["-std=c99", "-x", "c"]), ("g++", ["-std=c++17", "-x", "c++"])):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not available")
        r = subprocess.run([cc, *args, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", HEADER],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
