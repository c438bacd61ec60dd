"""Seeded procedural triangle meshes (FP64 construction, FP32 output).

Everything here builds *inputs*: vertex/triangle arrays, per-triangle material
and instance labels.  Nothing in this module computes any part of the LiDAR
model itself (no ray casting, shading, noise or cut-offs), so both the CUDA
path and the CPU oracle may consume its arrays.
"""
from __future__ import annotations

import numpy as np


class MeshBuilder:
    """Accumulates triangles; each add_* call appends one labelled part."""

    def __init__(self):
        self._verts = []
        self._tris = []
        self._mat = []
        self._inst = []
        self._nv = 0

    def add(self, verts64: np.ndarray, tris: np.ndarray, material, instance: int):
        verts64 = np.asarray(verts64, dtype=np.float64).reshape(-1, 3)
        tris = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
        self._verts.append(verts64.astype(np.float32))
        self._tris.append((tris + self._nv).astype(np.uint32))
        m = np.broadcast_to(np.asarray(material, dtype=np.uint16), (tris.shape[0],))
        self._mat.append(np.array(m, dtype=np.uint16))
        self._inst.append(np.full(tris.shape[0], instance, dtype=np.uint32))
        self._nv += verts64.shape[0]

    def build(self):
        verts = np.ascontiguousarray(np.concatenate(self._verts, axis=0), dtype=np.float32)
        tris = np.ascontiguousarray(np.concatenate(self._tris, axis=0), dtype=np.uint32)
        mat = np.ascontiguousarray(np.concatenate(self._mat), dtype=np.uint16)
        inst = np.ascontiguousarray(np.concatenate(self._inst), dtype=np.uint32)
        return verts, tris, mat, inst


# ---------------------------------------------------------------- primitives

def unit_box_faces(subdiv: int):
    """Unit cube [-0.5, 0.5]^3, each face split into subdiv x subdiv quads,
    two triangles per quad, counter-clockwise seen from outside."""
    verts, tris = [], []
    g = np.linspace(-0.5, 0.5, subdiv + 1)
    # each face: (normal axis, sign); tangent axes chosen so (t1 x t2) = +normal*sign
    for axis in range(3):
        for sign in (-1.0, 1.0):
            a1, a2 = (axis + 1) % 3, (axis + 2) % 3
            if sign < 0:
                a1, a2 = a2, a1
            base = len(verts)
            for j in range(subdiv + 1):
                for i in range(subdiv + 1):
                    p = [0.0, 0.0, 0.0]
                    p[axis] = 0.5 * sign
                    p[a1] = g[i]
                    p[a2] = g[j]
                    verts.append(p)
            for j in range(subdiv):
                for i in range(subdiv):
                    v00 = base + j * (subdiv + 1) + i
                    v10 = v00 + 1
                    v01 = v00 + (subdiv + 1)
                    v11 = v01 + 1
                    tris.append([v00, v10, v11])
                    tris.append([v00, v11, v01])
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int64)


def icosphere(subdiv: int):
    """Unit icosphere: icosahedron with each face split in four `subdiv` times,
    vertices projected onto the unit sphere, outward CCW winding."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]]
    f = [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [tuple(x) for x in f]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, dtype=np.int64)


def rot_z(yaw: float) -> np.ndarray:
    c, s = np.cos(yaw), np.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_y(pitch: float) -> np.ndarray:
    c, s = np.cos(pitch), np.sin(pitch)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def grid_terrain(n_cells: int, half_extent: float, height_fn):
    """Heightfield over [-half_extent, half_extent]^2 with n_cells^2 square cells,
    each split along the same diagonal into two CCW (seen from +z) triangles."""
    g = np.linspace(-half_extent, half_extent, n_cells + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")  # row = iy, col = ix
    Z = height_fn(X, Y)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    n1 = n_cells + 1
    iy, ix = np.meshgrid(np.arange(n_cells), np.arange(n_cells), indexing="ij")
    v00 = (iy * n1 + ix).ravel()
    v10 = v00 + 1
    v01 = v00 + n1
    v11 = v01 + 1
    tris = np.empty((2 * v00.size, 3), dtype=np.int64)
    tris[0::2] = np.stack([v00, v10, v11], axis=1)
    tris[1::2] = np.stack([v00, v11, v01], axis=1)
    return verts, tris, (ix.ravel(), iy.ravel())


class ValueNoiseFBM:
    """Fractional Brownian motion over 2-D value noise: per octave a lattice of
    uniform random values with smoothstep-blended bilinear interpolation."""

    def __init__(self, rng, half_extent, octaves=6, base_wavelength=128.0,
                 lacunarity=2.0, gain=0.5, amplitude=5.0):
        self.half = float(half_extent)
        self.octaves = []
        wl, amp = base_wavelength, 1.0
        for _ in range(octaves):
            n = int(np.ceil(2 * self.half / wl)) + 2
            self.octaves.append((wl, amp, rng.uniform(-1.0, 1.0, size=(n, n))))
            wl /= lacunarity
            amp *= gain
        # normalise so that max |h| over a probe grid equals `amplitude`
        probe = np.linspace(-self.half, self.half, 257)
        PX, PY = np.meshgrid(probe, probe)
        self.scale = 1.0
        m = np.abs(self.raw(PX, PY)).max()
        self.scale = amplitude / m if m > 0 else 1.0

    def raw(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        h = np.zeros(np.broadcast(x, y).shape)
        for wl, amp, lat in self.octaves:
            gx = (x + self.half) / wl
            gy = (y + self.half) / wl
            ix = np.clip(np.floor(gx).astype(np.int64), 0, lat.shape[1] - 2)
            iy = np.clip(np.floor(gy).astype(np.int64), 0, lat.shape[0] - 2)
            fx = gx - ix
            fy = gy - iy
            sx = fx * fx * (3 - 2 * fx)
            sy = fy * fy * (3 - 2 * fy)
            a = lat[iy, ix] * (1 - sx) + lat[iy, ix + 1] * sx
            b = lat[iy + 1, ix] * (1 - sx) + lat[iy + 1, ix + 1] * sx
            h = h + amp * (a * (1 - sy) + b * sy)
        return h * self.scale

    def __call__(self, x, y):
        return self.raw(x, y)
