"""gs_render_forward (eq. front-to-back, App. C rules) vs the FP64 oracle's per-pixel
definition: image, final transmittance and last contributor, element by element on every
pixel; where a decision lies within its margin of a threshold, the oracle's alternative with
that decision flipped is accepted too (gpu_util.compare_images)."""
import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import compare_images, gpu_forward

pytestmark = pytest.mark.gpu


def _cfg_pair(tile, mode="two_phase", batch=None):
    from paper_2308_04079_gb300 import make_config
    return make_config(tile=tile, sort_mode=mode, batch_depth=batch), oracle.cfg_array(tile_w=tile[0], tile_h=tile[1])


TINY = [
    (201, dict(n=200, width=100, height=37)),
    (202, dict(n=400, width=64, height=64, deg=0)),
    (203, dict(n=300, width=81, height=47, deg=2, log_scale_mean=-2.0)),
    (204, dict(n=600, width=130, height=70, deg=3, log_scale_mean=-3.0, opacity_logit_std=2.5)),
]


@pytest.mark.parametrize("tile", [(16, 16), (16, 8), (8, 8)])
@pytest.mark.parametrize("seed,kw", TINY)
def test_tiny_scenes(seed, kw, tile):
    g, cam = S.tiny_scene(seed, **kw)
    bg = (0.2, 0.4, 0.6)
    gcfg, ocfg = _cfg_pair(tile)
    run = gpu_forward(g, cam, bg, gcfg)
    orc = oracle.render_forward(g, cam, bg, ocfg)
    compare_images(run, orc, label=f"tiny{seed} {tile[0]}x{tile[1]}")


@pytest.mark.parametrize("mode,batch", [("two_phase", None), ("key64", None), ("two_phase", 32), ("key64", 100)])
def test_config1(mode, batch):
    """1,000 Gaussians, SH degree 0, 128x128, black background (config 1)."""
    g, cam, bg = S.config1()
    gcfg, ocfg = _cfg_pair((16, 16), mode, batch)
    run = gpu_forward(g, cam, bg, gcfg)
    orc = oracle.render_forward(g, cam, bg, ocfg)
    compare_images(run, orc, label=f"config1 {mode} batch {batch}")
    assert (run["last"] > 0).mean() > 0.3


def test_config2_full_frame():
    """200k Gaussians, SH degree 3, 1920x1080 (config 2), every pixel."""
    g, cam, bg, _ = S.config2()
    gcfg, ocfg = _cfg_pair((16, 16))
    run = gpu_forward(g, cam, bg, gcfg)
    orc = oracle.render_forward(g, cam, bg, ocfg)
    st = compare_images(run, orc, label="config2 1080p full frame")
    assert st["flagged_frac"] < 0.05


def test_config3_full_frame():
    """3M Gaussians, 1920x1080 (config 3, the benchmarked frame): every pixel of the frame,
    including the ragged bottom row of tiles, against the oracle."""
    g, cam, bg, _ = S.config3()
    gcfg, ocfg = _cfg_pair((16, 16))
    run = gpu_forward(g, cam, bg, gcfg)
    orc = oracle.render_forward(g, cam, bg, ocfg)
    st = compare_images(run, orc, label="config3 1080p full frame")
    assert st["flagged_frac"] < 0.05
    assert (run["last"] > 0).mean() > 0.2


def test_forward_is_deterministic():
    g, cam, bg, _ = S.config2(n=50_000)
    a = gpu_forward(g, cam, bg)
    b = gpu_forward(g, cam, bg)
    assert np.array_equal(a["img"], b["img"]) and np.array_equal(a["last"], b["last"])


@pytest.mark.parametrize("mode", ["two_phase", "key64"])
def test_reach_rule_renders_exactly_the_rectangle_image(mode):
    """The reachable-tile rule drops only (splat, tile) pairs whose alpha stays below 1/255 at
    every pixel of the tile: image, transmittance and last contributor are bit-identical to
    the paper's rectangle binning, with far fewer instances."""
    from paper_2308_04079_gb300 import make_config
    g, cam, bg, _ = S.config2()
    a = gpu_forward(g, cam, bg, make_config(sort_mode=mode, tile_rule="reach"))
    b = gpu_forward(g, cam, bg, make_config(sort_mode=mode, tile_rule="rect"))
    assert np.array_equal(a["img"], b["img"])
    assert np.array_equal(a["T"], b["T"])
    assert np.array_equal(a["last_id"], b["last_id"])
    ka = a["frame"].status()[1].num_instances
    kb = b["frame"].status()[1].num_instances
    assert ka < 0.75 * kb, (ka, kb)
