"""The bounds-checked build (-DLIDAR_BOUNDS, compute-sanitizer being closed on
this pool): every traversal tests each node and triangle index against its
array before reading it and reports a bad one in the status word.  On valid
scenes it must change nothing: every traversal variant, with and without
sub-rays, gives bit for bit the records of the normal build and a clean
status.  The checked library runs in a child process (one library per
process)."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import synth
from gpu_util import gpu_cast

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKLOADS = {
    "plain": dict(seed=3, n_frames=2, n_az=256),
    "subrays": dict(seed=9, n_frames=2, n_az=128, n_subrays=7, divergence=2e-3),
}
TRAVERSALS = (0, 1, 2, 3)

CHILD = textwrap.dedent("""
    import sys, numpy as np
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    from paper_2208_10295_gb300 import build, capi
    capi.load(build.build_checked())
    import synth
    from gpu_util import gpu_cast
    from paper_2208_10295_gb300 import Lidar
    L = Lidar(0)
    out = {{}}
    for name, kw in {workloads!r}.items():
        w = synth.small_terrain(**kw)
        scene = None
        for tv in {traversals!r}:
            L.set_launch_config(traversal=tv)
            g, scene = gpu_cast(L, w, scene)
            assert L.sync_status() == 0
            for k, v in g.items():
                out[f"{{name}}|{{tv}}|{{k}}"] = v
    np.savez({path!r}, **out)
    print("checked build ok")
""")


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


def test_checked_build_changes_nothing_on_valid_scenes(L, tmp_path):
    path = str(tmp_path / "checked.npz")
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), workloads=WORKLOADS,
                        traversals=TRAVERSALS, path=path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = np.load(path)
    cfg0 = L.launch_config()
    try:
        for name, kw in WORKLOADS.items():
            w = synth.small_terrain(**kw)
            scene = None
            for tv in TRAVERSALS:
                L.set_launch_config(traversal=tv)
                g, scene = gpu_cast(L, w, scene)
                for k, v in g.items():
                    assert np.array_equal(v.view(np.uint8), got[f"{name}|{tv}|{k}"].view(np.uint8)), (name, tv, k)
    finally:
        L.set_launch_config(**cfg0)
