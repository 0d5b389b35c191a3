"""Multi-scene batches: several scenes, each seen from several views, rendered forward and
backward as one FrameBatch (one launch per kernel for all frames), the whole step captured in
one CUDA graph, and an autotuner that picks the tile shape and the per-tile batch depth.

The rasterizer's arithmetic is the single-frame one: a batch changes how the work is launched,
never what a frame computes.  Each scene's gradients are the sum over its views."""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _abi as abi
from .rasterizer import Frame, FrameBatch, GaussianTensors, make_config

# Tile shapes and per-tile batch depths the autotuner tries (batch depth <= pixels per tile).
TILE_SHAPES = ((16, 16), (16, 8), (8, 8))
BATCH_DEPTHS = (32, 64, 128, 256)


@dataclass
class Scene:
    gaussians: GaussianTensors
    cameras: list
    dL_dimages: list           # per view, CUDA tensors [3, H, W]


class SceneBatch:
    """All views of all scenes as one batch; ``step()`` runs preprocess, binning, forward and
    backward once, ``capture()`` records that step in a CUDA graph and ``replay()`` re-runs it."""

    def __init__(self, scenes: list, bg=(0.0, 0.0, 0.0), cfg: abi.gs_raster_config | None = None,
                 headroom: float = 1.15):
        self.scenes = scenes
        self.bg = tuple(float(x) for x in bg)
        self.cfg = cfg if cfg is not None else make_config()
        views = [(s, cam, d) for s in scenes for cam, d in zip(s.cameras, s.dL_dimages)]
        if not 1 <= len(views) <= abi.GS_MAX_BATCH:
            raise ValueError(f"a batch holds 1..{abi.GS_MAX_BATCH} frames, got {len(views)}")
        frames = [Frame(s.gaussians.n, cam, self.cfg, device=d.device) for s, cam, d in views]
        probe = FrameBatch(frames, [s.gaussians for s, _, _ in views])
        probe.ensure_binned()
        # size every workspace to its measured instance count plus headroom
        self.frames = [Frame(s.gaussians.n, cam, self.cfg,
                             capacity=int(f.last_status.num_instances * headroom) + 4096, device=d.device)
                       for (s, cam, d), f in zip(views, frames)]
        del probe, frames
        self.batch = FrameBatch(self.frames, [s.gaussians for s, _, _ in views])
        self.dl = [d for _, _, d in views]
        self.outs = self.batch.outputs()
        self.grads = {id(s): self.frames[0].new_grads(s.gaussians) for s in scenes}
        self.view_grads = [self.grads[id(s)] for s, _, _ in views]
        self.graph = None

    def step(self) -> None:
        b = self.batch
        b.preprocess()
        b.bin_sort()
        b.render_forward(self.bg, self.outs)
        b.render_backward(self.bg, self.dl, self.outs, self.view_grads)

    def check(self) -> None:
        """Raise if any frame overflowed its capacity or timed out (synchronises)."""
        for f in self.frames:
            code, _ = f.status()
            if code not in (abi.GS_OK, abi.GS_ERR_NUMERIC):
                raise abi.GSError(code, "multi-scene step")

    def capture(self, warmup: int = 2) -> None:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(side)
        self.check()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()

    def replay(self) -> None:
        self.graph.replay()

    def time_replay(self, steps: int = 5) -> float:
        """Mean milliseconds per replayed step (CUDA events on the current stream)."""
        stream = torch.cuda.current_stream()
        self.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            self.replay()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    def scene_grads(self, scene: Scene) -> dict:
        return self.grads[id(scene)]


def candidates(tile_shapes=TILE_SHAPES, batch_depths=BATCH_DEPTHS):
    return [(t, b) for t in tile_shapes for b in batch_depths if b <= t[0] * t[1]]


def autotune(scenes: list, bg=(0.0, 0.0, 0.0), cands=None, steps: int = 3, sort_mode: str = "two_phase"):
    """Time the captured multi-scene step for every (tile shape, batch depth) candidate and
    return (best config, [(tile, batch_depth, ms), ...]).  Tile shapes are searched first at
    their largest batch depth, then the batch depth at the best tile shape."""
    cands = cands if cands is not None else candidates()
    shapes = sorted({t for t, _ in cands}, key=lambda t: -t[0] * t[1])
    table = []

    def measure(tile, depth):
        cfg = make_config(tile=tile, batch_depth=depth, sort_mode=sort_mode)
        sb = SceneBatch(scenes, bg, cfg)
        sb.capture()
        ms = sb.time_replay(steps)
        sb.check()
        del sb
        torch.cuda.empty_cache()
        table.append((tile, depth, ms))
        return ms

    best_shape, best_ms = None, float("inf")
    for t in shapes:
        depth = max(b for tt, b in cands if tt == t)
        ms = measure(t, depth)
        if ms < best_ms:
            best_shape, best_ms, best_depth = t, ms, depth
    for tt, b in cands:
        if tt == best_shape and b != best_depth:
            ms = measure(tt, b)
            if ms < best_ms:
                best_ms, best_depth = ms, b
    return make_config(tile=best_shape, batch_depth=best_depth, sort_mode=sort_mode), table
