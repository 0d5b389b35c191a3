"""Batched stages (gs_batch_*): several frames -- views of uneven size of one scene, or views
of several scenes -- in one launch per kernel.  Every frame's binning, image, transmittance and
last contributor equal the single-frame calls bit for bit; each scene's gradients equal the
per-view calls accumulated over its views (summation order differs: fp32 tolerance); the
config-4 batch (1M Gaussians, 16 uneven views) is checked against the FP64 oracle on every
pixel of every view and every Gaussian of the summed gradient, and the full-size config-5
multi-scene graph against the plain calls and, on sampled tiles, against the oracle."""
import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import compare_grads, compare_images, last_contributor_ids, oracle_view_sum

pytestmark = pytest.mark.gpu

GRAD_KEYS = ("means", "scales", "quats", "opacities", "sh", "mean2d")


def _single(gt, cams, bg, dimgs, cfg):
    """Per-view loop through the single-frame API, gradients accumulated over the views."""
    import torch
    from paper_2308_04079_gb300 import Frame
    outs, frames = [], []
    grads = None
    for v, cam in enumerate(cams):
        fr = Frame(gt.n, cam, cfg)
        fr.ensure_binned(gt)
        o = fr.outputs()
        fr.render_forward(bg, *o)
        if grads is None:
            grads = fr.new_grads(gt)
        fr.render_backward(gt, bg, dimgs[v], o[1], o[2], grads, accumulate=v > 0)
        outs.append(o)
        frames.append(fr)
    torch.cuda.synchronize()
    return frames, outs, grads


def _batched(groups, bg, cfg):
    """groups: list of (GaussianTensors, cams, dimgs) -> per-view frames/outs, per-group grads."""
    import torch
    from paper_2308_04079_gb300 import Frame, FrameBatch
    frames, gauss, dl, gr, grads = [], [], [], [], []
    for gt, cams, dimgs in groups:
        gd = None
        for cam, d in zip(cams, dimgs):
            fr = Frame(gt.n, cam, cfg)
            frames.append(fr)
            gauss.append(gt)
            dl.append(d)
            if gd is None:
                gd = fr.new_grads(gt)
                grads.append(gd)
            gr.append(gd)
    b = FrameBatch(frames, gauss)
    b.ensure_binned()
    outs = b.outputs()
    b.render_forward(bg, outs)
    b.render_backward(bg, dl, outs, gr)
    torch.cuda.synchronize()
    return frames, outs, grads


def _views(seed, n, views):
    import torch
    from paper_2308_04079_gb300 import GaussianTensors
    g, cams, _, dimgs = S.config4(k=seed, n=n, views=views)
    gt = GaussianTensors.from_numpy(g).prepared()
    return g, gt, cams, [torch.from_numpy(d).cuda() for d in dimgs]


def _assert_close_grads(a, b, what):
    """Batched vs per-view gradients: the screen-space accumulators are float atomics whose
    order differs run to run, so sums with cancellation differ in their last bits; per tensor
    relative L2 <= 1e-4, per element <= 1e-2 max(|g|, rms(g))."""
    a = a.astype(np.float64).reshape(a.shape[0], -1)
    b = b.astype(np.float64).reshape(b.shape[0], -1)
    na = np.linalg.norm(a)
    assert np.linalg.norm(a - b) <= 1e-4 * max(na, 1e-30), what
    rms = np.sqrt(np.mean(a ** 2)) if a.size else 0.0
    assert np.all(np.abs(a - b) <= 1e-2 * np.maximum(np.abs(a), rms) + 1e-30), what


def _assert_same_frame(fa, oa, fb, ob):
    import torch
    _, sa = fa.status()
    _, sb = fb.status()
    assert sa.num_instances == sb.num_instances and sa.num_visible == sb.num_visible
    K = int(sa.num_instances)
    for name, dt, cnt in (("vals_sorted", torch.int32, K), ("ranges", torch.int32, 2 * fa.tiles)):
        assert torch.equal(fa.view(name, dt, cnt), fb.view(name, dt, cnt)), name
    for x, y in zip(oa, ob):
        assert torch.equal(x, y)


@pytest.mark.parametrize("mode", ["two_phase", "key64"])
def test_batched_views_equal_per_view_calls(mode):
    import torch
    from paper_2308_04079_gb300 import make_config
    cfg = make_config(sort_mode=mode)
    _, gt, cams, dimgs = _views(7, 150_000, 6)
    bg = (0.1, 0.2, 0.3)
    fs, os_, gs = _single(gt, cams, bg, dimgs, cfg)
    fb, ob, gb = _batched([(gt, cams, dimgs)], bg, cfg)
    for v in range(len(cams)):
        _assert_same_frame(fs[v], os_[v], fb[v], ob[v])
    for k in GRAD_KEYS:
        _assert_close_grads(gs[k].cpu().numpy(), gb[0][k].cpu().numpy(), k)


def test_batched_scenes_keep_their_gradients_apart():
    """Three scenes of different sizes, two or three views each, in one batch."""
    import torch
    from paper_2308_04079_gb300 import make_config
    cfg = make_config()
    bg = (0.0, 0.0, 0.0)
    groups, singles = [], []
    for s, (n, views) in enumerate(((20_000, 2), (90_000, 3), (45_000, 2))):
        _, gt, cams, dimgs = _views(20 + s, n, views)
        groups.append((gt, cams, dimgs))
        singles.append(_single(gt, cams, bg, dimgs, cfg))
    fb, ob, gb = _batched(groups, bg, cfg)
    v = 0
    for s, (fs, os_, gs) in enumerate(singles):
        for k in range(len(fs)):
            _assert_same_frame(fs[k], os_[k], fb[v], ob[v])
            v += 1
        for key in GRAD_KEYS:
            _assert_close_grads(gs[key].cpu().numpy(), gb[s][key].cpu().numpy(), f"scene {s} {key}")


def test_config4_batch_matches_the_oracle():
    """Config 4 in full: one 1M-Gaussian scene (config-3 distribution), 16 views of uneven size
    (640x480 to 1920x1080) in one batch, forward and backward with the gradients summed over the
    views; every pixel of every view and every Gaussian's summed gradient against the oracle."""
    import torch
    from paper_2308_04079_gb300 import GaussianTensors, make_config
    g, cams, bg, dimgs = S.config4()
    gt = GaussianTensors.from_numpy(g).prepared()
    fb, ob, gb = _batched([(gt, cams, [torch.from_numpy(d).cuda() for d in dimgs])], bg, make_config())
    for v, cam in enumerate(cams):
        orc = oracle.render_forward(g, cam, bg)
        last = ob[v][2].cpu().numpy()
        run = dict(img=ob[v][0].cpu().numpy().astype(np.float64), T=ob[v][1].cpu().numpy().astype(np.float64),
                   last_id=last_contributor_ids(fb[v], last))
        compare_images(run, orc, label=f"config4 view {v} {cam.width}x{cam.height}")
    total = oracle_view_sum(g, cams, dimgs, bg)
    got = {k: gb[0][k].cpu().numpy().astype(np.float64) for k in ("means", "scales", "quats", "opacities", "sh")}
    compare_grads(got, total, label="config4 16 views summed")


def test_multiscene_graph_with_autotuned_config_matches_plain_calls():
    """Config-5 form, reduced: three scenes of 20k-80k Gaussians, two views each, the whole
    forward+backward step captured in one CUDA graph at the tile shape and batch depth the
    autotuner picks; every scene's images equal the plain per-view calls at that config and
    its gradients equal their sum over views; replaying the graph reproduces the images."""
    import torch
    from paper_2308_04079_gb300 import GaussianTensors
    from paper_2308_04079_gb300.batching import Scene, SceneBatch, autotune
    raw, bg = S.config5(k=9, scenes=3, views=2, n_min=20_000, n_max=80_000)
    bg = tuple(float(x) for x in bg)
    scenes = [Scene(GaussianTensors.from_numpy(g).prepared(), cams, [torch.from_numpy(d).cuda() for d in dl])
              for g, cams, dl in raw]
    cfg, table = autotune(scenes, bg, cands=[((16, 16), 128), ((16, 8), 64), ((8, 8), 64), ((8, 8), 32)], steps=2)
    # every tile shape at its largest depth, then the other depths of the best shape
    assert {t for t, _, _ in table} == {(16, 16), (16, 8), (8, 8)} and all(ms > 0 for _, _, ms in table)
    best = min(table, key=lambda r: r[2])
    assert (cfg.tile_w, cfg.tile_h) == best[0] and cfg.batch_depth == best[1]
    sb = SceneBatch(scenes, bg, cfg)
    sb.capture()
    sb.replay()
    torch.cuda.synchronize()
    sb.check()
    first = [o[0].clone() for o in sb.outs]
    sb.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, o[0]) for a, o in zip(first, sb.outs))
    v = 0
    for sc in scenes:
        fs, os_, gs = _single(sc.gaussians, sc.cameras, bg, sc.dL_dimages, cfg)
        for k in range(len(fs)):
            for x, y in zip(os_[k], sb.outs[v]):
                assert torch.equal(x, y)
            v += 1
        for key in GRAD_KEYS:
            _assert_close_grads(gs[key].cpu().numpy(), sb.scene_grads(sc)[key].cpu().numpy(), key)


def test_config5_full_size_graph_matches_plain_calls_and_the_oracle():
    """Config 5 at full size: 8 cluster-mixture scenes of 50k-2M Gaussians, 4 views each at
    mixed resolutions, forward+backward captured in one CUDA graph at the autotuned tile shape
    and batch depth.  The graph's images equal the plain per-view calls bit for bit and each
    scene's gradients their sum over views; on 8 sampled tiles per view (dL/dpixel zero
    elsewhere), images and every scene's gradients against the oracle at that tile shape."""
    import torch
    from paper_2308_04079_gb300 import GaussianTensors
    from paper_2308_04079_gb300.batching import Scene, SceneBatch, autotune
    raw, bg = S.config5()
    bg = tuple(float(x) for x in bg)
    rng = np.random.default_rng(5555)
    # the tile shape is chosen first (on full dL/dpixel); the sampled tiles follow it
    scenes = [Scene(GaussianTensors.from_numpy(g).prepared(), cams, [torch.from_numpy(d).cuda() for d in dl])
              for g, cams, dl in raw]
    cfg, table = autotune(scenes, bg, cands=[((16, 16), 128), ((16, 8), 128), ((8, 8), 64)], steps=2)
    tw, th = cfg.tile_w, cfg.tile_h
    masks, pixs = [], []
    for si, (g, cams, dl) in enumerate(raw):
        mm, pp = [], []
        for v, cam in enumerate(cams):
            TX, TY = (cam.width + tw - 1) // tw, (cam.height + th - 1) // th
            m = np.zeros(TX * TY, np.uint8)
            m[rng.choice(TX * TY, 8, replace=False)] = 1
            pix = np.repeat(np.repeat(m.reshape(TY, TX), th, 0), tw, 1)[:cam.height, :cam.width].astype(bool)
            dl[v] = np.where(pix[None], dl[v], 0.0).astype(np.float32)
            mm.append(m)
            pp.append(pix)
        masks.append(mm)
        pixs.append(pp)
    scenes = [Scene(GaussianTensors.from_numpy(g).prepared(), cams, [torch.from_numpy(d).cuda() for d in dl])
              for g, cams, dl in raw]
    sb = SceneBatch(scenes, bg, cfg)
    sb.capture()
    sb.replay()
    torch.cuda.synchronize()
    sb.check()
    ocfg = oracle.cfg_array(tile_w=tw, tile_h=th)
    v = 0
    for si, ((g, cams, dl), sc) in enumerate(zip(raw, scenes)):
        fs, os_, gs = _single(sc.gaussians, sc.cameras, bg, sc.dL_dimages, cfg)
        for k, cam in enumerate(cams):
            for x, y in zip(os_[k], sb.outs[v]):
                assert torch.equal(x, y)
            orc = oracle.render_forward(g, cam, bg, ocfg, tile_mask=masks[si][k])
            last = sb.outs[v][2].cpu().numpy()
            run = dict(img=sb.outs[v][0].cpu().numpy().astype(np.float64),
                       T=sb.outs[v][1].cpu().numpy().astype(np.float64),
                       last_id=last_contributor_ids(sb.frames[v], last))
            compare_images(run, orc, mask=pixs[si][k], label=f"config5 scene {si} view {k} {tw}x{th}")
            v += 1
        got = sb.scene_grads(sc)
        for key in GRAD_KEYS:
            _assert_close_grads(gs[key].cpu().numpy(), got[key].cpu().numpy(), key)
        total = oracle_view_sum(g, cams, dl, bg, ocfg, masks[si])
        compare_grads({k: got[k].cpu().numpy().astype(np.float64) for k in ("means", "scales", "quats",
                                                                           "opacities", "sh")},
                      total, label=f"config5 scene {si} ({g.n} Gaussians, 4 views)")
