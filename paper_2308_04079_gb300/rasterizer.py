"""PyTorch front end of the sm_103a tile rasterizer.

PyTorch provides device memory (the caller-owned workspace and the output tensors), the
current CUDA stream and autograd; every step of Algorithm 2 and of the backward pass runs in
the kernels of libgs_gb300.so, reached through the C ABI binding in :mod:`._abi`.

* :class:`Frame` -- one workspace sized for (Gaussian count, camera, constants, instance
  capacity) and the four stage calls on it.
* :func:`render` -- preprocess + bin/sort + blend, growing the instance capacity if needed.
* :func:`rasterize` -- differentiable rendering through :class:`RasterizeFunction`.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi as abi

_TILE_RULES = {"reach": abi.GS_TILES_REACH, "rect": abi.GS_TILES_RECT}
_SORT_MODES = {"two_phase": abi.GS_SORT_TWO_PHASE, "key64": abi.GS_SORT_KEY64}


def make_config(tile=(16, 16), batch_depth: int | None = None, sort_mode: str = "two_phase",
                tile_rule: str = "reach", grad_limit: int = 0, isotropic: bool = False,
                **overrides) -> abi.gs_raster_config:
    """Rasterizer constants (paper defaults) with optional overrides.  grad_limit > 0 and
    isotropic select the ablation variants of Sec. 7.3 (Limited-BW with N = grad_limit, and
    one scale per Gaussian with no rotation)."""
    cfg = abi.gs_default_config()
    cfg.tile_w, cfg.tile_h = int(tile[0]), int(tile[1])
    cfg.batch_depth = int(batch_depth) if batch_depth else cfg.tile_w * cfg.tile_h
    cfg.sort_mode = _SORT_MODES[sort_mode]
    cfg.tile_rule = _TILE_RULES[tile_rule]
    cfg.grad_limit = int(grad_limit)
    cfg.isotropic = int(bool(isotropic))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def camera_struct(cam) -> abi.gs_camera:
    """gs_camera from any object with width, height, fx, fy, cx, cy, R (3x3), t (3), near."""
    c = abi.gs_camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, dtype=np.float64).reshape(9)
    t = np.asarray(cam.t, dtype=np.float64).reshape(3)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(t[k])
    c.near_z = float(getattr(cam, "near", 0.2))
    return c


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _prep(t: torch.Tensor | None, align: int = 4) -> torch.Tensor | None:
    if t is None:
        return None
    t = t.detach()
    if t.dtype != torch.float32:
        raise TypeError("rasterizer inputs must be float32")
    if not t.is_cuda:
        raise ValueError("rasterizer inputs must be CUDA tensors")
    t = t.contiguous()
    if t.data_ptr() % align:
        t = t.clone()
    return t


@dataclass
class GaussianTensors:
    means: torch.Tensor      # [N, 3]
    scales: torch.Tensor     # [N, 3] ([N] for an isotropic configuration)
    quats: torch.Tensor      # [N, 4] (None for an isotropic configuration)
    opacities: torch.Tensor  # [N]
    sh: torch.Tensor         # [N, D, 3]
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def prepared(self) -> "GaussianTensors":
        return GaussianTensors(_prep(self.means), _prep(self.scales), _prep(self.quats, 16), _prep(self.opacities),
                               _prep(self.sh), int(self.sh_degree))

    def struct(self) -> abi.gs_gaussians:
        g = abi.gs_gaussians()
        g.means, g.scales, g.quats = _ptr(self.means), _ptr(self.scales), _ptr(self.quats)
        g.opacities, g.sh = _ptr(self.opacities), _ptr(self.sh)
        g.n, g.sh_degree, g.sh_stride = self.n, int(self.sh_degree), int(self.sh.shape[1])
        return g

    @staticmethod
    def from_numpy(g, device="cuda") -> "GaussianTensors":
        def t(a):
            return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(device)
        quats = None if g.quats is None else t(g.quats)
        return GaussianTensors(t(g.means), t(g.scales), quats, t(g.opacities), t(g.sh), int(g.sh_degree))


class Frame:
    """Caller-owned device workspace for one camera and the stage calls of Algorithm 2."""

    def __init__(self, n: int, camera, cfg: abi.gs_raster_config | None = None, capacity: int | None = None,
                 device: str | torch.device = "cuda"):
        abi.load()
        self.camera = camera
        self.cfg = cfg if cfg is not None else make_config()
        self.n = int(n)
        self.device = torch.device(device)
        self.cam = camera_struct(camera)
        self._alloc(int(capacity) if capacity is not None else max(1 << 16, 4 * self.n))

    def _alloc(self, capacity: int):
        self.capacity = min(int(capacity), (1 << 30) - 1)
        size = abi.gs_workspace_size(self.n, self.cam.width, self.cam.height, self.capacity, self.cfg)
        if size == 0:
            raise ValueError("invalid frame description")
        self.ws = torch.empty(size, dtype=torch.uint8, device=self.device)
        self.layout = abi.gs_workspace_layout(self.n, self.cam.width, self.cam.height, self.capacity, self.cfg)
        self.ws[self.layout.status:self.layout.status + ctypes.sizeof(abi.gs_device_status)].zero_()
        self.frame = abi.gs_frame(self.n, self.cam, self.cfg, self.capacity, self.ws.data_ptr(), size)

    def set_camera(self, camera) -> None:
        """Another camera of the same image size (the workspace layout stays valid)."""
        cam = camera_struct(camera)
        if (cam.width, cam.height) != (self.cam.width, self.cam.height):
            raise ValueError("set_camera keeps the image size")
        self.camera, self.cam = camera, cam
        self.frame.cam = cam

    @property
    def width(self) -> int:
        return self.cam.width

    @property
    def height(self) -> int:
        return self.cam.height

    @property
    def tiles(self) -> int:
        return self.layout.tiles_x * self.layout.tiles_y

    def view(self, name: str, dtype: torch.dtype, count: int) -> torch.Tensor:
        """Tensor view of a named workspace sub-buffer (see gs_layout)."""
        off = getattr(self.layout, name)
        nbytes = count * torch.empty(0, dtype=dtype).element_size()
        return self.ws[off:off + nbytes].view(dtype)

    # ---- stages -------------------------------------------------------------------------
    def preprocess(self, g: GaussianTensors) -> None:
        abi.gs_preprocess(self.frame, g.struct(), _stream())

    def bin_sort(self) -> None:
        abi.gs_bin_sort(self.frame, _stream())

    def bin_sort_timed(self) -> list:
        """gs_bin_sort with each launch timed: [(label, ms), ...] (synchronises)."""
        return abi.gs_bin_sort_timed(self.frame, _stream())

    def render_forward(self, bg, out_rgb: torch.Tensor, out_T: torch.Tensor, out_last: torch.Tensor) -> None:
        abi.gs_render_forward(self.frame, bg, out_rgb.data_ptr(), out_T.data_ptr(), out_last.data_ptr(), _stream())

    def render_backward(self, g: GaussianTensors, bg, dL_drgb: torch.Tensor, T: torch.Tensor, last: torch.Tensor,
                        grads: dict, accumulate: bool = False) -> None:
        gr = abi.gs_gradients()
        gr.means, gr.scales, gr.quats = _ptr(grads["means"]), _ptr(grads["scales"]), _ptr(grads["quats"])
        gr.opacities, gr.sh, gr.mean2d = _ptr(grads["opacities"]), _ptr(grads["sh"]), _ptr(grads.get("mean2d"))
        abi.gs_render_backward(self.frame, g.struct(), bg, dL_drgb.data_ptr(), T.data_ptr(), last.data_ptr(), gr,
                               accumulate, _stream())

    def render_backward_tiles(self, bg, dL_drgb: torch.Tensor, T: torch.Tensor, last: torch.Tensor) -> None:
        abi.gs_render_backward_tiles(self.frame, bg, dL_drgb.data_ptr(), T.data_ptr(), last.data_ptr(), _stream())

    def render_backward_gaussians(self, g: GaussianTensors, grads: dict, accumulate: bool = False) -> None:
        gr = abi.gs_gradients()
        gr.means, gr.scales, gr.quats = _ptr(grads["means"]), _ptr(grads["scales"]), _ptr(grads["quats"])
        gr.opacities, gr.sh, gr.mean2d = _ptr(grads["opacities"]), _ptr(grads["sh"]), _ptr(grads.get("mean2d"))
        abi.gs_render_backward_gaussians(self.frame, g.struct(), gr, accumulate, _stream())

    def status(self):
        """(status code, gs_device_status); synchronises the current stream."""
        return abi.gs_read_status(self.frame, _stream())

    def outputs(self):
        H, W = self.height, self.width
        return (torch.empty((3, H, W), dtype=torch.float32, device=self.device),
                torch.empty((H, W), dtype=torch.float32, device=self.device),
                torch.empty((H, W), dtype=torch.int32, device=self.device))

    def new_grads(self, g: GaussianTensors, with_mean2d: bool = True) -> dict:
        d = dict(means=torch.empty_like(g.means), scales=torch.empty_like(g.scales),
                 quats=None if g.quats is None else torch.empty_like(g.quats),
                 opacities=torch.empty_like(g.opacities),
                 sh=torch.empty_like(g.sh))
        if with_mean2d:
            d["mean2d"] = torch.empty((g.n, 2), dtype=torch.float32, device=g.means.device)
        return d

    def ensure_binned(self, g: GaussianTensors) -> None:
        """preprocess + bin_sort; if the instance capacity was too small, grow it and redo."""
        self.preprocess(g)
        self.bin_sort()
        code, st = self.status()
        if code == abi.GS_ERR_CAPACITY:
            self._alloc(int(st.num_instances * 1.25) + 1024)
            self.preprocess(g)
            self.bin_sort()
            code, st = self.status()
        if code in (abi.GS_ERR_CAPACITY, abi.GS_ERR_TIMEOUT, abi.GS_ERR_INTERNAL):
            raise abi.GSError(code, "gs_bin_sort")
        self.last_status = st


def _gradients_struct(grads: dict) -> abi.gs_gradients:
    gr = abi.gs_gradients()
    gr.means, gr.scales, gr.quats = _ptr(grads["means"]), _ptr(grads["scales"]), _ptr(grads["quats"])
    gr.opacities, gr.sh, gr.mean2d = _ptr(grads["opacities"]), _ptr(grads["sh"]), _ptr(grads.get("mean2d"))
    return gr


class FrameBatch:
    """Several frames (views of one or more scenes) rendered with one launch per kernel:
    ``frames[v]`` renders ``gaussians[v]``.  Frames that render the same GaussianTensors and
    receive the same gradient dict have their gradients summed (see gs_batch_render_backward)."""

    def __init__(self, frames: list, gaussians: list):
        if not 1 <= len(frames) <= abi.GS_MAX_BATCH or len(frames) != len(gaussians):
            raise ValueError("a batch holds 1..32 frames, one GaussianTensors each")
        self.frames = frames
        self.gaussians = gaussians

    def _structs(self):
        return [f.frame for f in self.frames]

    def preprocess(self) -> None:
        abi.gs_batch_preprocess(self._structs(), [g.struct() for g in self.gaussians], _stream())

    def bin_sort(self) -> None:
        abi.gs_batch_bin_sort(self._structs(), _stream())

    def ensure_binned(self) -> None:
        """preprocess + bin_sort of every frame; frames whose capacity was too small grow and
        the batch is binned again."""
        for _ in range(2):
            self.preprocess()
            self.bin_sort()
            grown = False
            for f in self.frames:
                code, st = f.status()
                if code == abi.GS_ERR_CAPACITY:
                    f._alloc(int(st.num_instances * 1.25) + 1024)
                    grown = True
                elif code in (abi.GS_ERR_TIMEOUT, abi.GS_ERR_INTERNAL):
                    raise abi.GSError(code, "gs_batch_bin_sort")
                f.last_status = st
            if not grown:
                return
        raise abi.GSError(abi.GS_ERR_CAPACITY, "gs_batch_bin_sort")

    def outputs(self):
        return [f.outputs() for f in self.frames]

    def render_forward(self, bg, outs) -> None:
        """bg: per-view (r, g, b) or one triple for all; outs: per-view (rgb, T, last)."""
        bgs = self._bgs(bg)
        abi.gs_batch_render_forward(self._structs(), bgs, [o[0].data_ptr() for o in outs],
                                    [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs], _stream())

    def render_backward(self, bg, dL_drgb: list, outs, grads: list, accumulate: bool = False) -> None:
        """dL_drgb: per-view tensors; outs: the forward's per-view (rgb, T, last); grads:
        per-view gradient dicts (the same dict for views whose gradients are summed)."""
        abi.gs_batch_render_backward(self._structs(), [g.struct() for g in self.gaussians], self._bgs(bg),
                                     [d.data_ptr() for d in dL_drgb], [o[1].data_ptr() for o in outs],
                                     [o[2].data_ptr() for o in outs], [_gradients_struct(g) for g in grads],
                                     accumulate, _stream())

    def _bgs(self, bg):
        bg = list(bg)
        if len(bg) == 3 and not hasattr(bg[0], "__len__"):
            return [tuple(float(x) for x in bg)] * len(self.frames)
        return [tuple(float(x) for x in b) for b in bg]


def _cfg_bytes(cfg) -> bytes:
    return bytes(cfg if cfg is not None else make_config())


def _frame_for(frame: Frame | None, n: int, camera, cfg, device) -> Frame:
    """``frame`` made ready for (n Gaussians, camera, cfg), or a new Frame when its Gaussian
    count, image size or constants differ or its workspace still waits for a backward pass."""
    cam = camera_struct(camera)
    if (frame is None or frame.n != n or (frame.cam.width, frame.cam.height) != (cam.width, cam.height)
            or bytes(frame.cfg) != _cfg_bytes(cfg) or getattr(frame, "pending_backward", False)):
        return Frame(n, camera, cfg, device=device)
    frame.set_camera(camera)
    return frame


def render(g: GaussianTensors, camera, bg=(0.0, 0.0, 0.0), cfg=None, frame: Frame | None = None):
    """Forward render.  Returns (image [3,H,W], T_final [H,W], last [H,W] int32, frame); a
    given ``frame`` is reused (with this camera) when its size and constants fit."""
    g = g.prepared()
    frame = _frame_for(frame, g.n, camera, cfg, g.means.device)
    frame.ensure_binned(g)
    img, T, last = frame.outputs()
    frame.render_forward(bg, img, T, last)
    return img, T, last, frame


class RasterizeFunction(torch.autograd.Function):
    """image = Rasterize(means, scales, quats, opacities, sh) for one camera (Algorithm 2);
    backward through the Sec. 6 traversal and the App. A chain rule.  The workspace of a
    forward pass stays reserved for its backward pass (it holds the binned instances and the
    screen-space splats that the backward reads); a second forward before that backward gets a
    workspace of its own."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, settings):
        g = GaussianTensors(means, scales, quats, opacities, sh, settings["sh_degree"]).prepared()
        frame = _frame_for(settings.get("frame"), g.n, settings["camera"], settings.get("cfg"), g.means.device)
        settings["frame"] = frame
        frame.ensure_binned(g)
        img, T, last = frame.outputs()
        frame.render_forward(settings["bg"], img, T, last)
        frame.pending_backward = True
        ctx.frame = frame
        ctx.g = g
        ctx.bg = settings["bg"]
        ctx.settings = settings
        ctx.save_for_backward(T, last)
        return img

    @staticmethod
    def backward(ctx, dimg):
        T, last = ctx.saved_tensors
        g = ctx.g
        grads = ctx.frame.new_grads(g)
        ctx.frame.render_backward(g, ctx.bg, _prep(dimg), T, last, grads)
        ctx.frame.pending_backward = False
        ctx.settings["mean2d_grad"] = grads["mean2d"]
        return grads["means"], grads["scales"], grads["quats"], grads["opacities"], grads["sh"], None


def rasterize(means, scales, quats, opacities, sh, sh_degree: int, camera, bg=(0.0, 0.0, 0.0), cfg=None,
              settings: dict | None = None) -> torch.Tensor:
    """Differentiable render of one view; returns the image [3, H, W].  ``settings`` (a dict)
    may be reused across calls and views to keep the workspace: each call renders with its
    own camera, background and constants, and a call made before the previous call's backward
    pass gets a fresh workspace.  After backward it holds the view-space mean gradient under
    ``"mean2d_grad"``."""
    s = settings if settings is not None else {}
    s.update(sh_degree=int(sh_degree), camera=camera, bg=tuple(float(x) for x in bg), cfg=cfg)
    return RasterizeFunction.apply(means, scales, quats, opacities, sh, s)
