"""Training step around the rasterizer (Sec. 5.1, Algorithm 1): render the Gaussians'
activated parameters, L = (1 - lambda) L1 + lambda (1 - SSIM) against a target view,
back-propagate through the rasterizer, and update the raw parameters with Adam (sigmoid
opacities, exp scales, exponentially decaying position learning rate); with a DensityControl
attached, also the gradient statistics and the refinement of Sec. 5.2.  Every step runs in the
library's kernels: gs_preprocess, gs_bin_sort, gs_render_forward, gs_render_backward,
gs_loss_l1_dssim, gs_adam_step (and gs_density_stats, gs_densify, gs_opacity_reset)."""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _abi as abi
from .rasterizer import Frame, GaussianTensors, _ptr, _stream, make_config


class Loss:
    """L1 + D-SSIM of planar [3, H, W] images (gs_loss_l1_dssim) with its image gradient."""

    def __init__(self, width: int, height: int, lam: float = 0.2, device="cuda"):
        self.width, self.height, self.lam = int(width), int(height), float(lam)
        size = abi.gs_loss_workspace_size(self.width, self.height)
        if size == 0:
            raise ValueError("invalid image size")
        self.ws = torch.empty(size + 256, dtype=torch.uint8, device=device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_view = self.ws[off:off + size]
        self.out = torch.zeros(3, dtype=torch.float32, device=device)

    def __call__(self, img: torch.Tensor, target: torch.Tensor, dL_dimg: torch.Tensor) -> torch.Tensor:
        """Writes dL/dimg; returns the device tensor (L, L1, mean SSIM)."""
        abi.gs_loss_l1_dssim(img.data_ptr(), target.data_ptr(), self.width, self.height, self.lam,
                             self.ws_view.data_ptr(), self.ws_view.numel(), self.out.data_ptr(), dL_dimg.data_ptr(),
                             _stream())
        return self.out


def _logit(p):
    p = np.clip(np.asarray(p, np.float64), 1e-6, 1 - 1e-6)
    return np.log(p / (1 - p))


@dataclass
class GaussianModel:
    """Raw parameters (log scales, logit opacities), their activated copies and Adam moments."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    logit_opacities: torch.Tensor
    sh: torch.Tensor
    sh_degree: int
    scales: torch.Tensor = None
    opacities: torch.Tensor = None
    moments: dict = field(default_factory=dict)

    @staticmethod
    def from_numpy(g, device="cuda") -> "GaussianModel":
        """From activated parameters (scales > 0, opacities in (0, 1))."""
        def t(a):
            return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(device)
        m = GaussianModel(t(g.means), t(np.log(np.asarray(g.scales, np.float64))), t(g.quats),
                          t(_logit(g.opacities)), t(g.sh), int(g.sh_degree))
        m.scales = torch.exp(m.log_scales)
        m.opacities = torch.sigmoid(m.logit_opacities)
        for k in ("means", "log_scales", "quats", "logit_opacities", "sh"):
            p = getattr(m, k)
            m.moments[k] = (torch.zeros_like(p), torch.zeros_like(p))
        return m

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def gaussians(self, sh_degree: int | None = None) -> GaussianTensors:
        """The activated parameters as the rasterizer's input, rendered up to ``sh_degree`` (the
        buffer keeps all coefficients; the unused ones get zero gradient)."""
        deg = self.sh_degree if sh_degree is None else min(int(sh_degree), self.sh_degree)
        return GaussianTensors(self.means, self.scales, self.quats, self.opacities, self.sh, deg)


def position_lr(step: int, lr_init: float, lr_final: float, max_steps: int) -> float:
    """Exponential decay (log-linear interpolation) of the position learning rate."""
    t = min(max(step / max(max_steps, 1), 0.0), 1.0)
    return math.exp((1 - t) * math.log(lr_init) + t * math.log(lr_final))


# Learning rates of the synthetic training runs (the paper gives the schedule's form only).
DEFAULT_LR = dict(means=1.6e-4, means_final=1.6e-6, means_steps=30000, log_scales=5e-3, quats=1e-3,
                  logit_opacities=5e-2, sh=2.5e-3)


class Trainer:
    """One training iteration per call of step(camera, target): forward, loss, backward, Adam."""

    def __init__(self, model: GaussianModel, lr: dict | None = None, lam: float = 0.2, betas=(0.9, 0.999),
                 eps: float = 1e-15, cfg=None, bg=(0.0, 0.0, 0.0), density=None, sh_band_every: int = 0):
        """sh_band_every > 0: optimise only the zero-order SH band first and add one band every
        that many iterations (Sec. 7.1 uses 1000); 0: all bands from the start."""
        self.model = model
        self.density = density
        self.sh_band_every = int(sh_band_every)
        self.lr = dict(DEFAULT_LR, **(lr or {}))
        self.lam, self.betas, self.eps = float(lam), betas, float(eps)
        self.cfg = cfg if cfg is not None else make_config()
        self.bg = tuple(float(x) for x in bg)
        self.iteration = 0
        self._frames = {}
        self._loss = {}
        self.grads = None

    def _frame(self, camera) -> tuple:
        key = (camera.width, camera.height)
        if key not in self._frames:
            fr = Frame(self.model.n, camera, self.cfg, device=self.model.means.device)
            fr.ensure_binned(self.model.gaussians())
            fr = Frame(self.model.n, camera, self.cfg, capacity=int(fr.last_status.num_instances * 1.5) + 4096,
                       device=self.model.means.device)
            self._frames[key] = (fr, fr.outputs(), torch.empty((3, camera.height, camera.width),
                                                              dtype=torch.float32, device=self.model.means.device))
            self._loss[key] = Loss(camera.width, camera.height, self.lam, device=self.model.means.device)
        fr, outs, dimg = self._frames[key]
        fr.set_camera(camera)
        return fr, outs, dimg, self._loss[key]

    def step(self, camera, target: torch.Tensor) -> torch.Tensor:
        """Returns the device tensor (L, L1, mean SSIM) of this iteration's rendering."""
        m = self.model
        fr, (img, T, last), dimg, loss = self._frame(camera)
        g = m.gaussians(self.active_sh_degree())
        if self.grads is None:
            self.grads = fr.new_grads(g, with_mean2d=True)
        fr.preprocess(g)
        fr.bin_sort()
        fr.render_forward(self.bg, img, T, last)
        out = loss(img, target, dimg)
        fr.render_backward(g, self.bg, dimg, T, last, self.grads)
        if self.density is not None:
            self.density.accumulate(fr, self.grads["mean2d"])
        self.iteration += 1
        t = self.iteration
        lr = self.lr
        groups = []
        for name, grad_key, act, act_out, rate in (
                ("means", "means", abi.GS_ACT_NONE, None, position_lr(t - 1, lr["means"], lr["means_final"],
                                                                       lr["means_steps"])),
                ("log_scales", "scales", abi.GS_ACT_EXP, m.scales, lr["log_scales"]),
                ("quats", "quats", abi.GS_ACT_NONE, None, lr["quats"]),
                ("logit_opacities", "opacities", abi.GS_ACT_SIGMOID, m.opacities, lr["logit_opacities"]),
                ("sh", "sh", abi.GS_ACT_NONE, None, lr["sh"])):
            p = getattr(m, name)
            mm, vv = m.moments[name]
            grp = abi.gs_adam_group()
            grp.param, grp.grad, grp.m, grp.v = _ptr(p), _ptr(self.grads[grad_key]), _ptr(mm), _ptr(vv)
            grp.activated = _ptr(act_out) if act_out is not None else None
            grp.n, grp.lr, grp.activation = p.numel(), float(rate), act
            groups.append(grp)
        abi.gs_adam_step(groups, self.betas[0], self.betas[1], self.eps, t, _stream())
        if self.density is not None and self.density.after_step(t):
            self._frames.clear()      # workspaces and gradients are sized by the Gaussian count
            self.grads = None
        return out

    def active_sh_degree(self) -> int:
        """SH degree rendered at the next iteration under the band schedule."""
        if self.sh_band_every <= 0:
            return self.model.sh_degree
        return min(self.model.sh_degree, self.iteration // self.sh_band_every)

    def status(self):
        """Status codes of the frames (synchronises)."""
        return {k: v[0].status()[0] for k, v in self._frames.items()}
