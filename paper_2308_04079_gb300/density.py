"""Adaptive density control (Sec. 5.2, the refinement step of Algorithm 1) on the device.

DensityControl keeps the per-Gaussian view-space gradient statistics of a GaussianModel
(gs_density_stats after every backward pass), runs the refinement (gs_densify: prune, clone,
split in one compaction pass) on the schedule of Sec. 5.2 and resets the opacities
(gs_opacity_reset).  The host only sizes buffers and reads the new Gaussian count back.

Schedule and thresholds: the paper gives tau_pos = 0.0002, phi = 1.6, a refinement every 100
iterations after a warm-up and an opacity reset every 3000 iterations.  Its other constants
are unstated; the defaults here are readings: warm-up 500 iterations, refinement until
iteration 15000, epsilon_alpha = 0.005, tau_S = 0.01 x the scene extent, the world-size and
screen-size pruning (0.1 x extent, 20 px) active after the first opacity reset, reset opacity
0.01, scene extent = 1.1 x the largest distance of a training camera from the cameras' mean
centre (the distance of the camera from the origin when there is one camera)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _abi as abi
from .rasterizer import _ptr, _stream

PARAMS = ("means", "log_scales", "quats", "logit_opacities", "sh")


@dataclass
class DensitySchedule:
    start: int = 500              # first refinement after this many iterations
    every: int = 100              # Sec. 5.2
    stop: int = 15000             # no refinement after this iteration
    reset_every: int = 3000       # Sec. 5.2: opacity reset period
    reset_opacity: float = 0.01

    def refine_at(self, iteration: int) -> bool:
        return self.start < iteration <= self.stop and iteration % self.every == 0

    def reset_at(self, iteration: int) -> bool:
        return self.reset_every > 0 and iteration <= self.stop and iteration % self.reset_every == 0

    def size_pruning(self, iteration: int) -> bool:
        return self.reset_every > 0 and iteration > self.reset_every


def scene_extent(cameras) -> float:
    """1.1 x the largest distance of a camera centre (C = -R^T t) from the centres' mean."""
    centres = []
    for cam in cameras:
        R = np.asarray(cam.R, np.float64).reshape(3, 3)
        centres.append(-R.T @ np.asarray(cam.t, np.float64).reshape(3))
    c = np.stack(centres)
    radius = float(np.linalg.norm(c - c.mean(axis=0), axis=1).max())
    if radius == 0.0:
        radius = float(np.linalg.norm(c[0]))
    return 1.1 * radius


def _arrays(tensors: dict) -> abi.gs_param_arrays:
    p = abi.gs_param_arrays()
    p.means, p.log_scales, p.quats = _ptr(tensors["means"]), _ptr(tensors["log_scales"]), _ptr(tensors["quats"])
    p.logit_opacities, p.sh = _ptr(tensors["logit_opacities"]), _ptr(tensors["sh"])
    return p


class DensityControl:
    """Gradient statistics and refinement of one GaussianModel."""

    def __init__(self, model, extent: float, grad_threshold: float = 0.0002, min_opacity: float = 0.005,
                 split_fraction: float = 0.01, world_fraction: float = 0.1, max_screen_radius: float = 20.0,
                 split_factor: float = 1.6, schedule: DensitySchedule | None = None):
        self.model = model
        self.extent = float(extent)
        self.grad_threshold, self.min_opacity = float(grad_threshold), float(min_opacity)
        self.split_scale = float(split_fraction) * self.extent
        self.max_world_scale = float(world_fraction) * self.extent
        self.max_screen_radius = float(max_screen_radius)
        self.split_factor = float(split_factor)
        self.schedule = schedule or DensitySchedule()
        self.last_result = None
        self._zero_stats(model.n)

    def _zero_stats(self, n: int) -> None:
        dev = self.model.means.device
        self.grad_accum = torch.zeros(n, dtype=torch.float32, device=dev)
        self.grad_count = torch.zeros(n, dtype=torch.float32, device=dev)
        self.max_radius = torch.zeros(n, dtype=torch.float32, device=dev)

    def config(self, size_pruning: bool) -> abi.gs_density_config:
        c = abi.gs_density_config()
        c.grad_threshold, c.min_opacity, c.split_scale = self.grad_threshold, self.min_opacity, self.split_scale
        c.max_world_scale = self.max_world_scale if size_pruning else 0.0
        c.max_screen_radius = self.max_screen_radius if size_pruning else 0.0
        c.split_factor = self.split_factor
        return c

    def accumulate(self, frame, mean2d_grad: torch.Tensor) -> None:
        """Add one rendered view (its frame and the mean2d gradient of its backward pass)."""
        abi.gs_density_stats(frame.frame, _ptr(mean2d_grad), _ptr(self.grad_accum), _ptr(self.grad_count),
                             _ptr(self.max_radius), _stream())

    def refine(self, size_pruning: bool = False, generator: torch.Generator | None = None) -> int:
        """Prune, clone and split; replaces the model's tensors and moments.  Returns the new
        Gaussian count (synchronises once to read it)."""
        m = self.model
        n, dev = m.n, m.means.device
        cap = 2 * n
        sh_floats = m.sh[0].numel() if n else int(np.prod(m.sh.shape[1:]))
        normals = torch.randn((n, 2, 3), dtype=torch.float32, device=dev, generator=generator)
        out = {k: torch.empty((cap,) + tuple(getattr(m, k).shape[1:]), dtype=torch.float32, device=dev)
               for k in PARAMS}
        out_m = {k: torch.empty_like(out[k]) for k in PARAMS}
        out_v = {k: torch.empty_like(out[k]) for k in PARAMS}
        scales = torch.empty((cap, 3), dtype=torch.float32, device=dev)
        opac = torch.empty(cap, dtype=torch.float32, device=dev)
        stats = [torch.empty(cap, dtype=torch.float32, device=dev) for _ in range(3)]
        result = torch.zeros(2, dtype=torch.int32, device=dev)
        scratch_bytes = abi.gs_densify_scratch_size(n)
        scratch = torch.empty(scratch_bytes + 256, dtype=torch.uint8, device=dev)
        off = (-scratch.data_ptr()) % 256
        src = {k: getattr(m, k) for k in PARAMS}
        abi.gs_densify(self.config(size_pruning), n, sh_floats, _arrays(src),
                       _arrays({k: m.moments[k][0] for k in PARAMS}), _arrays({k: m.moments[k][1] for k in PARAMS}),
                       _ptr(self.grad_accum), _ptr(self.grad_count), _ptr(self.max_radius), _ptr(normals),
                       _arrays(out), _arrays(out_m), _arrays(out_v), _ptr(stats[0]), _ptr(stats[1]), _ptr(stats[2]),
                       _ptr(scales), _ptr(opac), cap, _ptr(result), scratch.data_ptr() + off, scratch_bytes,
                       _stream())
        count, flags = (int(x) for x in result.cpu())
        self.last_result = (count, flags)
        if flags:
            raise abi.GSError(abi.GS_ERR_TIMEOUT if flags & abi.FLAG_TIMEOUT else abi.GS_ERR_CAPACITY, "gs_densify")
        for k in PARAMS:
            setattr(m, k, out[k][:count])
            m.moments[k] = (out_m[k][:count], out_v[k][:count])
        m.scales, m.opacities = scales[:count], opac[:count]
        self.grad_accum, self.grad_count, self.max_radius = (t[:count] for t in stats)
        return count

    def reset_opacity(self) -> None:
        m = self.model
        mm, vv = m.moments["logit_opacities"]
        abi.gs_opacity_reset(_ptr(m.logit_opacities), _ptr(mm), _ptr(vv), _ptr(m.opacities), m.n,
                             self.schedule.reset_opacity, _stream())

    def after_step(self, iteration: int) -> bool:
        """Run what the schedule asks for after optimiser step `iteration`; True when the
        Gaussian count may have changed."""
        changed = False
        if self.schedule.refine_at(iteration):
            self.refine(size_pruning=self.schedule.size_pruning(iteration))
            changed = True
        if self.schedule.reset_at(iteration):
            self.reset_opacity()
        return changed
