"""Treelet restructuring of the binary hierarchy (Karras and Aila, HPG 2013).

Checked against what the surface-area model fixes, not against the kernel's
own dynamic program: on scenes of up to seven triangles one round makes the
whole tree a single treelet, so its cost must equal the cheapest of every
binary tree over those triangles, found here by enumerating all of them; on a
larger scene the rounds must not raise the cost; and the closest hits (every
dense field of the full cfg1 frame and of a terrain with sub-rays) must not
change at all, whichever tree is walked."""
import json

import numpy as np
import pytest

import synth
from gpu_util import gpu_cast, setup

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _half_area(lo, hi, w=(1.0, 1.0, 1.0)):
    """Half the surface of a box with its faces normal to x, y, z weighted by
    w (1, 1, 1: half the surface area)."""
    d = np.asarray(hi, np.float64) - np.asarray(lo, np.float64)
    return w[2] * d[0] * d[1] + w[0] * d[1] * d[2] + w[1] * d[2] * d[0]


def _child_boxes(b):
    """(lo, hi) of the left and right child of one exported binary node."""
    return ((np.array([b[0], b[2], b[8]]), np.array([b[1], b[3], b[9]])),
            (np.array([b[4], b[6], b[10]]), np.array([b[5], b[7], b[11]])))


def _check_binary_tree(nodes, leaf_tri, verts, tris, w=(1.0, 1.0, 1.0)):
    """Every triangle once, every node but the root once, each stored child box
    the exact FP32 box of what lies below; returns the leaf-ordered triangle
    boxes and the sum of the internal nodes' (weighted) half areas (FP64)."""
    n = tris.shape[0]
    assert nodes.shape[0] == n - 1
    assert np.array_equal(np.sort(leaf_tri), np.arange(n))
    V = verts[tris[leaf_tri]]
    lo_t, hi_t = V.min(1), V.max(1)
    child = nodes[:, 12:14].view(np.int32)
    seen_leaf = np.zeros(n, int)
    seen_node = np.zeros(n - 1, int)
    box = {}

    def box_of(c):
        if c < 0:
            return lo_t[~c], hi_t[~c]
        if c not in box:
            (a_lo, a_hi), (b_lo, b_hi) = _child_boxes(nodes[c])
            box[c] = (np.minimum(a_lo, b_lo), np.maximum(a_hi, b_hi))
        return box[c]

    inner = 0.0
    for i in range(n - 1):
        lo_i, hi_i = box_of(i)
        inner += _half_area(lo_i, hi_i, w)
        for side, (lo, hi) in enumerate(_child_boxes(nodes[i])):
            c = int(child[i, side])
            if c < 0:
                seen_leaf[~c] += 1
            else:
                seen_node[c] += 1
            clo, chi = box_of(c)
            assert np.array_equal(lo, clo) and np.array_equal(hi, chi), (i, side)
    assert np.all(seen_leaf == 1)
    assert seen_node[0] == 0 and np.all(seen_node[1:] == 1)
    return lo_t, hi_t, inner


def _all_tree_costs(boxes, w=(1.0, 1.0, 1.0)):
    """Sum of the internal nodes' (weighted) half areas of every binary tree
    over the given leaf boxes (each unordered tree once: the first leaf of a
    set always goes to the first part)."""
    def union(S):
        lo = np.min([boxes[i][0] for i in S], axis=0)
        hi = np.max([boxes[i][1] for i in S], axis=0)
        return _half_area(lo, hi, w)

    def costs(S):
        if len(S) == 1:
            yield 0.0
            return
        a = union(S)
        first, rest = S[0], S[1:]
        for mask in range(1 << len(rest)):
            P = (first,) + tuple(r for j, r in enumerate(rest) if mask >> j & 1)
            Q = tuple(r for j, r in enumerate(rest) if not mask >> j & 1)
            if not Q:
                continue
            qs = list(costs(Q))
            for cp in costs(P):
                for cq in qs:
                    yield a + cp + cq

    return costs(tuple(range(len(boxes))))


def _random_triangles(n, seed):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-10.0, 10.0, (n, 1, 3))
    verts = (centres + rng.uniform(-1.5, 1.5, (n, 3, 3))).reshape(-1, 3).astype(np.float32)
    tris = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
    return verts, tris


@pytest.mark.parametrize("w", [(1.0, 1.0, 1.0), (1.0, 0.5, 0.23)])
@pytest.mark.parametrize("n", [3, 4, 5, 6, 7])
def test_one_round_gives_the_cheapest_tree_of_up_to_seven_triangles(L, n, w):
    counts = {}
    try:
        for seed in range(4):
            verts, tris = _random_triangles(n, 100 * n + seed)
            for method in (0, 1):
                L.set_build_options(method=method, treelet_rounds=1, area_weight=w)
                scene = L.build_scene(verts, tris)
                nodes, leaf_tri = scene.export()
                lo_t, hi_t, inner = _check_binary_tree(nodes, leaf_tri, verts, tris, w)
                best = min(_all_tree_costs(list(zip(lo_t, hi_t)), w))
                # FP32 costs in the kernel, and a rewrite only when the optimum is
                # cheaper by more than 1e-5 relative
                assert inner <= best * (1.0 + 3e-5), (n, seed, method, inner, best)
                counts[f"seed{seed}_m{method}"] = scene.info()["treelets"]
                scene.free()
    finally:
        L.set_build_options(method=1, treelet_rounds=0, area_weight=(1.0, 1.0, 1.0))
    print(json.dumps({"label": f"{n} triangles, face weights {w}: treelets rewritten", **counts}))


@pytest.mark.parametrize("aw", [(1.0, 1.0, 1.0), (1.0, 1.0, 0.23)])
def test_rounds_never_raise_the_tree_cost(L, aw):
    w = synth.small_terrain(seed=8, n_cells=48, half=24.0, n_objects=20, n_frames=1, n_az=32)
    verts, tris = w.scene.verts, w.scene.tris
    res = {}
    try:
        for method in (0, 1):
            prev = None
            for rounds in (0, 1, 2, 3):
                L.set_build_options(method=method, treelet_rounds=rounds, area_weight=aw)
                scene = L.build_scene(verts, tris, w.scene.mat, w.scene.inst)
                nodes, leaf_tri = scene.export()
                _, _, inner = _check_binary_tree(nodes, leaf_tri, verts, tris, aw)
                info = scene.info()
                assert info["max_depth"] <= 96
                if rounds == 0:
                    assert info["treelets"] == 0
                else:
                    assert info["treelets"] > 0
                    assert inner <= prev * (1.0 + 1e-6), (method, rounds, inner, prev)
                res[(method, rounds)] = inner
                prev = inner
                scene.free()
    finally:
        L.set_build_options(method=1, treelet_rounds=0, area_weight=(1.0, 1.0, 1.0))
    # the rounds lower the cost of the Karras tree (splits at Morton bits, not by area)
    assert res[(0, 3)] < 0.99 * res[(0, 0)]
    print(json.dumps({"label": f"small terrain internal-node area sums, face weights {aw}",
                      **{f"m{m}_r{r}": v for (m, r), v in res.items()}}))


def test_treelet_trees_cast_bit_identical(L):
    """Every dense field of the full cfg1 frame, of a small terrain with
    sub-rays and of one city frame (7 sub-rays per beam), bit for bit, through
    both wide traversals, on the plain PLOC tree, with two treelet rounds, and
    on the benchmark's trees (treelet rounds and face-weighted areas): the
    closest hit does not depend on the hierarchy."""
    from bench import CFG1_TREE, CITY_TREE
    fields = ("valid", "tri", "t", "range", "intensity", "normal", "mat", "inst", "theta_deg")
    plain = dict(treelet_rounds=0, area_weight=(1.0, 1.0, 1.0))
    cfg0 = L.launch_config()
    out = {}
    try:
        city = synth.cfg4()
        city.frames = city.frames[1:2]
        for w in (synth.cfg1(), synth.small_terrain(seed=9, n_frames=2, n_az=128, n_subrays=7, divergence=2e-3),
                  city):
            trees = [dict(treelet_rounds=2, area_weight=(1.0, 1.0, 1.0)), CITY_TREE if w is city else CFG1_TREE]
            for tv in ((2, 3) if w is not city else (2,)):
                L.set_launch_config(traversal=tv)
                L.set_build_options(method=1, **plain)
                base, s0 = gpu_cast(L, w, fields=fields)
                fetches = [L.count_work(s0, w.frames, w.seed)["node_visits"]] if tv == 2 else []
                s0.free()
                for tree in trees:
                    L.set_build_options(method=1, **tree)
                    other, s1 = gpu_cast(L, w, fields=fields)
                    for k in fields:
                        assert np.array_equal(base[k].view(np.uint8), other[k].view(np.uint8)), (w.name, tv, tree, k)
                    if tv == 2:
                        fetches.append(L.count_work(s1, w.frames, w.seed)["node_visits"])
                    s1.free()
                if tv == 2:
                    n = L.total_beams(w.frames)
                    out[w.name] = [f / n for f in fetches]
    finally:
        L.set_build_options(method=1, **plain)
        L.set_launch_config(**cfg0)
    print(json.dumps({"label": "4-wide node fetches per ray: plain PLOC, 2 treelet rounds, the benchmark's tree",
                      **out}))


def test_wide_trees_of_a_restructured_tree(L):
    """The 4- and 8-wide trees collapsed from a restructured binary tree (face-
    weighted areas) hold every triangle once, with exact boxes."""
    w = synth.small_terrain(seed=8, n_cells=48, half=24.0, n_objects=20, n_frames=1, n_az=32)
    try:
        L.set_build_options(method=1, treelet_rounds=3, area_weight=(1.0, 1.0, 0.23))
        scene, _ = setup(L, w)
    finally:
        L.set_build_options(method=1, treelet_rounds=0, area_weight=(1.0, 1.0, 1.0))
    _, leaf_tri = scene.export()
    V = w.scene.verts[w.scene.tris[leaf_tri]]
    lo_t, hi_t = V.min(1).astype(np.float32), V.max(1).astype(np.float32)
    from test_gpu_parity import _wide_tree_invariants
    for width in (4, 8):
        _wide_tree_invariants(scene.export_wide(width), width, w.scene.n_tris, lo_t, hi_t)
    scene.free()
