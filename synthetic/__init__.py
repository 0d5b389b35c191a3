"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests, the smoke
check and the benchmark.  This package holds input generation only (scene
distributions, camera poses, upstream gradients) and none of the rasterizer's
arithmetic; it imports neither the oracle nor the CUDA path."""
from .scenes import (Camera, Gaussians, look_at_camera, orbit_camera, config1, config2, config2_crop,
                     config3, config4, config5, density_state, tiny_scene, upstream_grad)

__all__ = ["Camera", "Gaussians", "look_at_camera", "orbit_camera", "config1", "config2", "config2_crop",
           "config3", "config4", "config5", "density_state", "tiny_scene", "upstream_grad"]
