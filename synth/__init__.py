"""Seeded synthetic inputs for the LiDAR return-generation path.

This package only *draws* inputs (scenes, beam patterns, trajectories,
material parameters).  It contains none of the method's arithmetic, so the
CUDA path and the CPU oracle can both consume what it produces.
"""
from .geometry import MeshBuilder, ValueNoiseFBM, icosphere, unit_box_faces  # noqa: F401
from .sensors import (SensorSpec, material_params, raster_pattern, sensor_16ch,  # noqa: F401
                      sensor_32ch, sensor_64ch, sensor_128ch, sensor_raster, spinning_pattern)
from .workloads import (FRAME_DTYPE, SWEEP_FRAME_DTYPE, make_sweep_frames, Scene, Workload, by_index, cfg0, cfg1, cfg2, cfg3,  # noqa: F401
                        cfg4, make_frames, pose_rows, small_terrain, adjoint_tape)
