"""gs_render_backward (Sec. 6 traversal, App. A chain rule) vs the oracle's analytic FP64
gradients, for the screen-space accumulators and for every input tensor; the oracle's
analytic gradients are themselves pinned to finite differences on the CPU.  Every Gaussian is
checked: the per-element bound holds exactly, plus, for a Gaussian that a decision near its
threshold touches, the oracle's allowance for that decision being flipped."""
import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import compare_grads, gpu_backward, gpu_forward

pytestmark = pytest.mark.gpu


def _check(g, cam, bg, dimg, tile_mask=None, cfg=None, label="", ocfg=None):
    run = gpu_forward(g, cam, bg, cfg)
    gg = gpu_backward(run, bg, dimg)
    ob = oracle.render_backward(g, cam, dimg, bg, cfg=ocfg, tile_mask=tile_mask)
    assert ob["dec_overflow"] == 0
    touched = np.abs(ob["opacities"]) > 0
    assert touched.sum() > 10
    ob2 = dict(ob)
    ob2["opac2d"] = ob["opacities"]
    s2 = compare_grads(gg, ob2, names=("uv", "cov2d", "opac2d", "rgb"), label=label + " screen space")
    s3 = compare_grads(gg, ob, label=label)
    return s2, s3


@pytest.mark.parametrize("seed,kw", [(301, dict(n=200, width=100, height=37)),
                                     (302, dict(n=300, width=64, height=64, deg=0)),
                                     (303, dict(n=400, width=90, height=70, deg=3, log_scale_mean=-3.0)),
                                     (304, dict(n=300, width=48, height=48, deg=1, opacity_logit_std=2.5))])
def test_tiny_scene_gradients(seed, kw):
    g, cam = S.tiny_scene(seed, **kw)
    dimg = S.upstream_grad(seed + 1, cam.height, cam.width)
    _check(g, cam, (0.1, 0.3, 0.2), dimg, label=f"tiny{seed}")


@pytest.mark.parametrize("tile", [(16, 8), (8, 8)])
@pytest.mark.parametrize("seed,kw", [(301, dict(n=200, width=100, height=37)),
                                     (303, dict(n=400, width=90, height=70, deg=3, log_scale_mean=-3.0))])
def test_tiny_scene_gradients_other_tile_shapes(seed, kw, tile):
    """The 16x8 and 8x8 tile shapes (one warp per tile; two pixels per thread for 8x8): the
    oracle bins with the same shape (the 3-sigma rectangle is tile-granular, so the shape is
    part of the definition)."""
    from paper_2308_04079_gb300 import make_config
    g, cam = S.tiny_scene(seed, **kw)
    dimg = S.upstream_grad(seed + 1, cam.height, cam.width)
    _check(g, cam, (0.1, 0.3, 0.2), dimg, cfg=make_config(tile=tile),
           ocfg=oracle.cfg_array(tile_w=tile[0], tile_h=tile[1]), label=f"tiny{seed} {tile[0]}x{tile[1]}")


def test_config2_crop_gradients():
    """The config-2 gradient-check case: 5k Gaussians, 64x64 window of the 1080p camera."""
    g, cam, bg, dimg = S.config2_crop()
    _check(g, cam, bg, dimg, label="config2 64x64 crop")


def test_config2_full_frame_gradients():
    g, cam, bg, dimg = S.config2()
    _check(g, cam, bg, dimg, label="config2 1080p full frame")


def test_config3_full_frame_gradients():
    """3M Gaussians at 1080p (config 3, the benchmarked frame): dL/dpixel ~ N(0, 1) on every
    pixel, all gradients of all 3M Gaussians against the oracle."""
    g, cam, bg, dimg = S.config3()
    _check(g, cam, bg, dimg, label="config3 1080p full frame")


def test_accumulate_over_views_sums_gradients():
    import torch
    g, cam1 = S.tiny_scene(305, n=200, width=64, height=48)
    cam2 = S.orbit_camera(3.0, 0.4, 0.2, 64, 48)
    d1, d2 = S.upstream_grad(1, 48, 64), S.upstream_grad(2, 48, 64)
    bg = (0.0, 0.0, 0.0)
    r1, r2 = gpu_forward(g, cam1, bg), gpu_forward(g, cam2, bg)
    g1, g2 = gpu_backward(r1, bg, d1), gpu_backward(r2, bg, d2)
    # accumulate view 2 into view 1's gradients
    from paper_2308_04079_gb300 import GaussianTensors
    grads = {k: torch.from_numpy(v.astype(np.float32)).cuda() for k, v in g1.items()
             if k in ("means", "scales", "quats", "opacities", "sh", "mean2d")}
    r2["frame"].render_backward(r2["g"], bg, torch.from_numpy(d2).cuda(), r2["T_t"], r2["last_t"], grads,
                                accumulate=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        np.testing.assert_allclose(grads[k].cpu().numpy(), g1[k] + g2[k], rtol=1e-5, atol=1e-6)


def test_autograd_function_matches_direct_calls():
    import torch
    from paper_2308_04079_gb300 import rasterize
    g, cam = S.tiny_scene(306, n=200, width=64, height=48)
    dimg = S.upstream_grad(7, 48, 64)
    bg = (0.1, 0.1, 0.1)
    t = {k: torch.tensor(getattr(g, k), device="cuda", requires_grad=True)
         for k in ("means", "scales", "quats", "opacities", "sh")}
    img = rasterize(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], g.sh_degree, cam, bg)
    (img * torch.from_numpy(dimg).cuda()).sum().backward()
    run = gpu_forward(g, cam, bg)
    direct = gpu_backward(run, bg, dimg)
    np.testing.assert_array_equal(img.detach().cpu().numpy(), run["img"].astype(np.float32))
    for k in t:
        np.testing.assert_allclose(t[k].grad.cpu().numpy(), direct[k], rtol=1e-5, atol=1e-7)


def test_autograd_settings_reused_across_views_match_fresh_calls():
    """One settings dict reused for two cameras (one of another image size), and two forward
    passes before their backward passes: every image and gradient equals a fresh call's."""
    import torch
    from paper_2308_04079_gb300 import rasterize
    g, cam1 = S.tiny_scene(307, n=250, width=64, height=48)
    cam2 = S.orbit_camera(3.0, 0.6, -0.2, 64, 48)
    cam3 = S.orbit_camera(3.0, -0.4, 0.3, 80, 40)
    bg = (0.2, 0.1, 0.3)

    def params():
        return {k: torch.tensor(getattr(g, k), device="cuda", requires_grad=True)
                for k in ("means", "scales", "quats", "opacities", "sh")}

    def run(cam, settings=None):
        t = params()
        img = rasterize(t["means"], t["scales"], t["quats"], t["opacities"], t["sh"], g.sh_degree, cam, bg,
                        settings=settings)
        return t, img

    fresh = {}
    for name, cam in (("1", cam1), ("2", cam2), ("3", cam3)):
        t, img = run(cam)
        d = torch.from_numpy(S.upstream_grad(int(name), cam.height, cam.width)).cuda()
        (img * d).sum().backward()
        fresh[name] = (img.detach().clone(), {k: v.grad.clone() for k, v in t.items()}, d)
    shared = {}
    # sequential reuse across cameras and image sizes
    for name, cam in (("1", cam1), ("2", cam2), ("3", cam3)):
        t, img = run(cam, shared)
        (img * fresh[name][2]).sum().backward()
        assert torch.equal(img.detach(), fresh[name][0]), name
        for k in t:
            torch.testing.assert_close(t[k].grad, fresh[name][1][k], rtol=1e-5, atol=1e-7)
    # two forward passes on one settings dict before either backward pass
    ta, ia = run(cam1, shared)
    tb, ib = run(cam2, shared)
    (ib * fresh["2"][2]).sum().backward()
    (ia * fresh["1"][2]).sum().backward()
    for (t, img), name in (((ta, ia), "1"), ((tb, ib), "2")):
        assert torch.equal(img.detach(), fresh[name][0]), name
        for k in t:
            torch.testing.assert_close(t[k].grad, fresh[name][1][k], rtol=1e-5, atol=1e-7)
