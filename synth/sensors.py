"""Beam patterns (the paper's per-beam spherical coordinates, azimuth theta_i and
elevation phi_j, Sec. II-A) and sensor constants, as plain input data.

Azimuth is measured in the sensor's x-y plane from +x towards +y; elevation
from that plane towards +z.  Spinning patterns are ordered column-major: all
channels of one azimuth step are consecutive (beam = az_index * n_ch + ch),
which is the order a spinning LiDAR fires them.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class SensorSpec:
    name: str
    az_rad: np.ndarray          # float64 [B]
    el_rad: np.ndarray          # float64 [B]
    r_min: float = 0.5
    r_max: float = 100.0
    d_max: float = 100.0        # capability model maximum range (Eq. 5)
    RL_max: float = 0.80        # reflectance needed at d_max (Eq. 5), as a fraction
    sigma: float = 0.02         # Gaussian range-noise standard deviation [m]
    gain: float = 1.0
    range_exp: float = 0.0      # p in I = g R (r_ref/d)^p; 0 = the paper's intensity
    r_ref: float = 1.0
    divergence_rad: float = 0.0  # full beam divergence; 0 = single ray per beam
    n_subrays: int = 1
    sigma_k: float = 0.0        # range-scaled noise: std = sigma + sigma_k * t

    @property
    def n_beams(self) -> int:
        return int(self.az_rad.shape[0])


def spinning_pattern(elev_deg, n_az: int):
    el = np.deg2rad(np.asarray(elev_deg, dtype=np.float64))
    az = 2.0 * np.pi * np.arange(n_az, dtype=np.float64) / n_az
    AZ = np.repeat(az, el.size)
    EL = np.tile(el, n_az)
    return np.ascontiguousarray(AZ), np.ascontiguousarray(EL)


def raster_pattern(width: int, height: int, fov_h_deg: float, fov_v_deg: float):
    """Solid-state raster: pixel centres on a regular (azimuth, elevation) grid,
    row-major with elevation rows from bottom to top."""
    i = np.arange(width, dtype=np.float64)
    j = np.arange(height, dtype=np.float64)
    az = np.deg2rad(-fov_h_deg / 2 + (i + 0.5) * fov_h_deg / width)
    el = np.deg2rad(-fov_v_deg / 2 + (j + 0.5) * fov_v_deg / height)
    EL, AZ = np.meshgrid(el, az, indexing="ij")
    return np.ascontiguousarray(AZ.ravel()), np.ascontiguousarray(EL.ravel())


def elevations_16ch():
    return -15.0 + 2.0 * np.arange(16)


def elevations_32ch():
    return -16.0 + 1.0 * np.arange(32)


def elevations_64ch():
    return np.linspace(-25.0, 15.0, 64)


def elevations_128ch():
    """Non-uniform 128-channel layout: 0.1 deg spacing within +-2 deg of the
    horizon, coarser below (-25..-2.4) and above (+2.4..+15)."""
    fine = np.round(np.arange(-20, 21) * 0.1, 10)            # 41 channels
    low = -25.0 + np.arange(56) * 23.0 / 56.0                 # 56 channels
    high = 2.0 + np.arange(1, 32) * 13.0 / 31.0               # 31 channels
    e = np.concatenate([low, fine, high])
    assert e.size == 128
    return e


def sensor_16ch(n_az=1800, **kw):
    az, el = spinning_pattern(elevations_16ch(), n_az)
    return SensorSpec("spin16", az, el, **kw)


def sensor_32ch(n_az=2048, **kw):
    az, el = spinning_pattern(elevations_32ch(), n_az)
    return SensorSpec("spin32", az, el, **kw)


def sensor_64ch(n_az=2048, **kw):
    az, el = spinning_pattern(elevations_64ch(), n_az)
    return SensorSpec("spin64", az, el, **kw)


def sensor_128ch(n_az=2048, **kw):
    az, el = spinning_pattern(elevations_128ch(), n_az)
    return SensorSpec("spin128", az, el, **kw)


def sensor_raster(width=256, height=128, fov_h=120.0, fov_v=25.0, **kw):
    az, el = raster_pattern(width, height, fov_h, fov_v)
    return SensorSpec("raster256x128", az, el, **kw)


def material_params(rng, n_materials: int) -> np.ndarray:
    """Per-material (a, s, w_deg): Lambertian albedo a ~ U[0.05, 0.9], specular
    lobe height s ~ U[0, min(0.5, 1-a)] and width w ~ U[2, 10] degrees."""
    a = rng.uniform(0.05, 0.9, size=n_materials)
    w = rng.uniform(2.0, 10.0, size=n_materials)
    s = rng.uniform(0.0, 1.0, size=n_materials) * np.minimum(0.5, 1.0 - a)
    return np.ascontiguousarray(np.stack([a, s, w], axis=1).astype(np.float32))
