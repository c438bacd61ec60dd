"""GB300-native per-beam LiDAR return generation ("Physical LiDAR Simulation in
Real-Time Engine", Sec. II) behind the C ABI of include/lidar.h.

    capi       ctypes binding, same names as the C ABI
    torch_api  tensor-level wrapper (Lidar, Scene), the LidarCast autograd Function and the
               combination of sharded fused-MSE adjoints (combine_mse, allreduce_mse)
    build      compiles csrc/*.cu for sm_103a into _build/liblidar.so
"""
from . import capi  # noqa: F401

__all__ = ["capi", "build_library", "Lidar", "LidarCast"]


def build_library(force: bool = False) -> str:
    from .build import build
    return build(force=force)


def __getattr__(name):
    if name in ("Lidar", "LidarCast", "Scene", "FRAME_DTYPE", "combine_mse", "allreduce_mse"):
        from . import torch_api
        return getattr(torch_api, name)
    raise AttributeError(name)
