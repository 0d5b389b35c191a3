"""The ablation variants of Sec. 7.3 on the CUDA path against the oracle: Limited-BW
(cfg.grad_limit = N: gradients only for each pixel's N front-most blended splats, image
unchanged) and isotropic Gaussians (cfg.isotropic: one scale per Gaussian, no rotation)."""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import compare_grads, compare_images, gpu_backward, gpu_forward

pytestmark = pytest.mark.gpu


def _cfg(**kw):
    from paper_2308_04079_gb300 import make_config
    return make_config(**kw)


def _grads_vs_oracle(g, cam, bg, dimg, cfg, ocfg, iso=False, label=""):
    run = gpu_forward(g, cam, bg, cfg)
    gg = gpu_backward(run, bg, dimg)
    f = oracle.render_backward_isotropic if iso else oracle.render_backward
    ob = f(g, cam, dimg, bg, ocfg)
    assert ob["dec_overflow"] == 0
    touched = np.abs(ob["opacities"]) > 0
    assert touched.sum() > 20
    names = ("means", "scales", "opacities", "sh") if iso else ("means", "scales", "quats", "opacities", "sh")
    compare_grads(gg, ob, names=names, label=label)
    return run, gg, ob


@pytest.mark.parametrize("N", [10, 1, 3])
def test_limited_bw_gradients_match_the_oracle(N):
    g, cam = S.tiny_scene(401, n=1500, width=120, height=90, deg=3, log_scale_mean=-2.6, opacity_logit_std=0.8)
    dimg = S.upstream_grad(402, cam.height, cam.width)
    bg = (0.1, 0.2, 0.3)
    run, gg, ob = _grads_vs_oracle(g, cam, bg, dimg, _cfg(grad_limit=N), oracle.cfg_array(grad_limit=N),
                                   label=f"Limited-BW N={N}")
    if N < 10:   # a tight limit takes gradients away: some Gaussians the full gradient reaches get none
        full = oracle.render_backward(g, cam, dimg, bg)
        assert (np.abs(full["opacities"]) > 0).sum() > (np.abs(ob["opacities"]) > 0).sum()


def test_limited_bw_leaves_the_image_unchanged_and_a_deep_limit_is_the_full_gradient():
    g, cam = S.tiny_scene(403, n=800, width=96, height=64, deg=2)
    dimg = S.upstream_grad(404, cam.height, cam.width)
    bg = (0.0, 0.0, 0.0)
    plain = gpu_forward(g, cam, bg)
    lim = gpu_forward(g, cam, bg, _cfg(grad_limit=10))
    assert np.array_equal(plain["img"], lim["img"]) and np.array_equal(plain["last"], lim["last"])
    deep = gpu_forward(g, cam, bg, _cfg(grad_limit=100000))
    a, b = gpu_backward(plain, bg, dimg), gpu_backward(deep, bg, dimg)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-5, atol=1e-6 * np.abs(a[k]).max())


def test_limited_bw_config2_crop():
    g, cam, bg, dimg = S.config2_crop()
    _grads_vs_oracle(g, cam, bg, dimg, _cfg(grad_limit=10), oracle.cfg_array(grad_limit=10),
                     label="Limited-BW N=10 config2 crop")


def _iso(g):
    n = g.means.shape[0]
    s = np.exp(np.log(np.asarray(g.scales, np.float64)).mean(axis=1)).astype(np.float32)
    return SimpleNamespace(means=g.means, scales=s, quats=None, opacities=g.opacities, sh=g.sh,
                           sh_degree=g.sh_degree, n=n)


@pytest.mark.parametrize("seed,kw", [(411, dict(n=600, width=100, height=70, deg=3)),
                                     (412, dict(n=300, width=64, height=40, deg=0, log_scale_mean=-2.0))])
def test_isotropic_image_and_gradients_match_the_oracle(seed, kw):
    g, cam = S.tiny_scene(seed, **kw)
    gi = _iso(g)
    bg = (0.2, 0.1, 0.0)
    cfg = _cfg(isotropic=True)
    run = gpu_forward(gi, cam, bg, cfg)
    compare_images(run, oracle.render_forward_isotropic(gi, cam, bg), label=f"isotropic tiny{seed}")
    dimg = S.upstream_grad(seed + 1, cam.height, cam.width)
    run, gg, ob = _grads_vs_oracle(gi, cam, bg, dimg, cfg, None, iso=True, label=f"isotropic tiny{seed}")
    assert gg["scales"].shape == (gi.n,) and "quats" not in gg


def test_variants_in_a_batch_equal_single_frames():
    """Two views rendered as one batch with both variants on: images and summed gradients equal
    the two single-frame calls."""
    import torch
    from paper_2308_04079_gb300 import Frame, FrameBatch, GaussianTensors
    g, cam1 = S.tiny_scene(421, n=700, width=80, height=60, deg=3)
    cam2 = S.orbit_camera(3.0, 0.5, 0.1, 72, 56)
    gi = _iso(g)
    cfg = _cfg(grad_limit=5, isotropic=True)
    gt = GaussianTensors.from_numpy(gi).prepared()
    bg = (0.0, 0.0, 0.0)
    dl = [torch.from_numpy(S.upstream_grad(422 + k, c.height, c.width)).cuda() for k, c in enumerate((cam1, cam2))]
    # single frames, gradients accumulated over the two views
    single = {}
    for k, cam in enumerate((cam1, cam2)):
        fr = Frame(gt.n, cam, cfg)
        fr.ensure_binned(gt)
        img, T, last = fr.outputs()
        fr.render_forward(bg, img, T, last)
        gr = fr.new_grads(gt)
        fr.render_backward(gt, bg, dl[k], T, last, gr)
        torch.cuda.synchronize()
        single[k] = (img.cpu().numpy(), {n: v.cpu().numpy() for n, v in gr.items() if v is not None})
    frames = [Frame(gt.n, c, cfg) for c in (cam1, cam2)]
    fb = FrameBatch(frames, [gt, gt])
    fb.ensure_binned()
    outs = fb.outputs()
    fb.render_forward([bg, bg], outs)
    grads = frames[0].new_grads(gt)
    fb.render_backward([bg, bg], dl, outs, [grads, grads])
    torch.cuda.synchronize()
    for k in range(2):
        assert np.array_equal(outs[k][0].cpu().numpy(), single[k][0])
    for n, v in grads.items():
        if v is None:
            continue
        want = single[0][1][n] + single[1][1][n]
        got = v.cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-4 * max(np.linalg.norm(want), 1e-12), n
