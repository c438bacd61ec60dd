"""Hand-built tiny scenes and sensors for pins and edge cases (inputs only)."""
import numpy as np

from synth import Scene, SensorSpec, make_frames, pose_rows


def quads_scene(quads, materials=None, instances=None):
    """Each quad is 4 corner points (counter-clockwise); two triangles per quad."""
    verts, tris, mat, inst = [], [], [], []
    for k, q in enumerate(quads):
        base = 4 * k
        verts += list(q)
        tris += [[base, base + 1, base + 2], [base, base + 2, base + 3]]
        m = 0 if materials is None else materials[k]
        i = k if instances is None else instances[k]
        mat += [m, m]
        inst += [i, i]
    return Scene(np.array(verts, np.float32), np.array(tris, np.uint32), np.array(mat, np.uint16),
                 np.array(inst, np.uint32))


def ground_quad(half=1000.0, z=0.0):
    return [(-half, -half, z), (half, -half, z), (half, half, z), (-half, half, z)]


def wall_x(x, half=50.0):
    """Plane x = const facing -x."""
    return [(x, -half, -half), (x, -half, half), (x, half, half), (x, half, -half)]


def sensor(az, el, **kw):
    kw.setdefault("sigma", 0.0)
    return SensorSpec("test", np.asarray(az, np.float64), np.asarray(el, np.float64), **kw)


def identity_frame(origin=(0.0, 0.0, 0.0), frame=0):
    return make_frames([(0, frame, pose_rows(np.eye(3), origin))])


def const_table(c, M=1):
    return np.full((M, 91), float(c))


def random_tris_scene(rng, n=30, lo=2.0, hi=10.0, size=3.0):
    """Random triangles in a shell around the origin, plus a ground quad."""
    verts, tris = [], []
    for k in range(n):
        r = rng.uniform(lo, hi)
        az = rng.uniform(0, 2 * np.pi)
        el = rng.uniform(-0.6, 0.6)
        c = r * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        for _ in range(3):
            verts.append(c + rng.uniform(-size, size, 3))
        tris.append([3 * k, 3 * k + 1, 3 * k + 2])
    nv = len(verts)
    verts += [(-20, -20, -3), (20, -20, -3), (20, 20, -3), (-20, 20, -3)]
    tris += [[nv, nv + 1, nv + 2], [nv, nv + 2, nv + 3]]
    nt = len(tris)
    return Scene(np.array(verts, np.float32), np.array(tris, np.uint32),
                 (np.arange(nt) % 3).astype(np.uint16), np.arange(nt, dtype=np.uint32))
