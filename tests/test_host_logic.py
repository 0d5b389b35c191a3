"""Host-side logic of the training loop (no GPU): the density-control schedule of Sec. 5.2,
the scene extent, the progressive SH band schedule of Sec. 7.1 and the position learning
rate of the Trainer."""
import math
from types import SimpleNamespace

import numpy as np
import torch

from paper_2308_04079_gb300.density import DensitySchedule, scene_extent
from paper_2308_04079_gb300.training import GaussianModel, Trainer, position_lr
from synthetic import look_at_camera


def test_density_schedule():
    s = DensitySchedule()
    assert not s.refine_at(500) and s.refine_at(600) and not s.refine_at(650)
    assert s.refine_at(15000) and not s.refine_at(15100)
    assert s.reset_at(3000) and s.reset_at(6000) and not s.reset_at(3100) and not s.reset_at(18000)
    assert not s.size_pruning(3000) and s.size_pruning(3001)
    every = DensitySchedule(start=0, every=1, stop=10, reset_every=0)
    assert all(every.refine_at(i) for i in range(1, 11)) and not every.reset_at(3)


def test_scene_extent():
    cams = [look_at_camera([3.0 * math.cos(a), 0.0, 3.0 * math.sin(a)], [0, 0, 0], 64, 48, 60.0)
            for a in np.linspace(0, 2 * math.pi, 8, endpoint=False)]
    assert abs(scene_extent(cams) - 1.1 * 3.0) < 1e-5          # centres on a circle of radius 3
    one = [look_at_camera([0.0, 0.0, -4.0], [0, 0, 0], 64, 48, 60.0)]
    assert abs(scene_extent(one) - 1.1 * 4.0) < 1e-5           # one camera: its distance to the origin


def _model(n=5, deg=3):
    rng = np.random.default_rng(0)
    g = SimpleNamespace(means=rng.normal(size=(n, 3)), scales=np.full((n, 3), 0.1), quats=np.tile([1.0, 0, 0, 0], (n, 1)),
                        opacities=np.full(n, 0.5), sh=rng.normal(size=(n, (deg + 1) ** 2, 3)), sh_degree=deg)
    return GaussianModel.from_numpy(g, device="cpu")


def test_sh_band_schedule():
    m = _model()
    tr = Trainer(m, sh_band_every=1000)
    seen = []
    for it in (0, 999, 1000, 1999, 2000, 3000, 9000):
        tr.iteration = it
        seen.append(tr.active_sh_degree())
    assert seen == [0, 0, 1, 1, 2, 3, 3]
    assert Trainer(m).active_sh_degree() == 3
    assert m.gaussians(1).sh_degree == 1 and m.gaussians(7).sh_degree == 3 and m.gaussians().sh_degree == 3


def test_position_lr_is_log_linear():
    assert math.isclose(position_lr(0, 1.6e-4, 1.6e-6, 30000), 1.6e-4)
    assert math.isclose(position_lr(30000, 1.6e-4, 1.6e-6, 30000), 1.6e-6)
    assert math.isclose(position_lr(15000, 1.6e-4, 1.6e-6, 30000), 1.6e-5)
    assert math.isclose(position_lr(90000, 1.6e-4, 1.6e-6, 30000), 1.6e-6)


def test_bench_launch_count_and_byte_model_follow_the_schedule():
    """bench.py's kernel count per step and algorithmic binning bytes for the row-segmented tile
    sort (1080p, 16x16 tiles), the two-phase radix sort (over 255 tile columns) and KEY64,
    from the workspace layout the library reports."""
    import bench
    from paper_2308_04079_gb300 import _abi
    c = _abi.gs_default_config()
    rows = _abi.gs_workspace_layout(3_000_000, 1920, 1080, 1 << 20, c)
    wide = _abi.gs_workspace_layout(3_000_000, 4400, 1080, 1 << 20, c)
    c.sort_mode = _abi.GS_SORT_KEY64
    k64 = _abi.gs_workspace_layout(3_000_000, 1920, 1080, 1 << 20, c)
    assert bench.row_sort(rows) and not bench.row_sort(wide) and not bench.row_sort(k64)
    # preprocess, clear, depth histogram + 4 depth passes, segment pass, sort-prepare, row pass,
    # column count, tile scan, column pass, tile order, forward, clear, backward tiles, backward
    # Gaussians
    assert bench.launches_per_step(rows) == 18
    # the same with emit + 2 tile-id passes + ranges in place of the row sort's four kernels
    assert bench.launches_per_step(wide) == 1 + 1 + 5 + 1 + 1 + 1 + wide.key_passes + 1 + 1 + 4
    # KEY64: count + pair scan + segment write + emit + sort-prepare + 6 passes + ranges
    assert bench.launches_per_step(k64) == 1 + 1 + 3 + 3 + 6 + 1 + 4
    n, n_vis, K, segs, tiles = 3_000_000, 2_436_483, 28_516_288, 9_019_658, 8160
    depth = 8 * n + 4 * 16 * n
    b = bench.byte_model(n, n_vis, K, segs, 1920 * 1080, tiles, 48, rows)["bin_sort"]
    assert b == depth + n_vis * 44 + segs * (8 + 16 + 4 + 8) + tiles * 12 + K * 8
    b = bench.byte_model(n, n_vis, K, segs, 1920 * 1080, tiles, 48, wide)["bin_sort"]
    assert b == depth + n_vis * 44 + segs * 24 + K * 8 + 2 * 2 * K * 8 + tiles * 8
