"""Density-control kernels (Sec. 5.2) against the FP64 oracle, through the C ABI:
gs_densify (prune / clone / split compaction), gs_density_stats (view-space gradient
statistics of a rendered view) and gs_opacity_reset; and a training run that refines."""
import numpy as np
import pytest

import synthetic as S
from oracle import density as od

pytestmark = pytest.mark.gpu

PARAMS = od.PARAMS


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _arrays(t):
    from paper_2308_04079_gb300 import _abi
    p = _abi.gs_param_arrays()
    for k in PARAMS:
        setattr(p, k, t[k].data_ptr() if t[k].numel() else None)
    return p


def _config(c: od.DensityConfig):
    from paper_2308_04079_gb300 import _abi
    g = _abi.gs_density_config()
    for k in ("grad_threshold", "min_opacity", "split_scale", "max_world_scale", "max_screen_radius", "split_factor"):
        setattr(g, k, getattr(c, k))
    return g


def _gpu_densify(state, cfg: od.DensityConfig, capacity=None):
    """Run gs_densify on `state` (the tuple of synthetic.density_state); returns the outputs as
    numpy arrays cut to min(count, capacity) rows, the count, the flags and the zeroed stats."""
    import torch
    from paper_2308_04079_gb300 import _abi
    f, m, v, acc, cnt, mr, z = state
    n = f["means"].shape[0]
    cap = 2 * n if capacity is None else capacity
    src, sm, sv = ({k: _cuda(d[k]) for k in PARAMS} for d in (f, m, v))
    out, om, ov = ({k: torch.full((cap,) + f[k].shape[1:], np.nan, dtype=torch.float32, device="cuda")
                    for k in PARAMS} for _ in range(3))
    stats = [torch.full((cap,), 7.0, dtype=torch.float32, device="cuda") for _ in range(3)]
    scales = torch.full((cap, 3), np.nan, dtype=torch.float32, device="cuda")
    opac = torch.full((cap,), np.nan, dtype=torch.float32, device="cuda")
    result = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    sb = _abi.gs_densify_scratch_size(n)
    scratch = torch.empty(sb + 256, dtype=torch.uint8, device="cuda")
    off = (-scratch.data_ptr()) % 256
    ta, tc, tm, tz = _cuda(acc), _cuda(cnt), _cuda(mr), _cuda(z)
    sh_floats = int(np.prod(f["sh"].shape[1:]))
    _abi.gs_densify(_config(cfg), n, sh_floats, _arrays(src), _arrays(sm), _arrays(sv), ta.data_ptr() if n else None,
                    tc.data_ptr() if n else None, tm.data_ptr() if n else None, tz.data_ptr() if n else None,
                    _arrays(out), _arrays(om), _arrays(ov), *(s.data_ptr() if cap else None for s in stats),
                    scales.data_ptr() if cap else None, opac.data_ptr() if cap else None, cap, result.data_ptr(),
                    scratch.data_ptr() + off if n else None, sb, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    count, flags = (int(x) for x in result.cpu())
    k = min(count, cap)
    cut = lambda d: {key: t[:k].cpu().numpy() for key, t in d.items()}
    return (cut(out), cut(om), cut(ov), count, flags, [s[:k].cpu().numpy() for s in stats],
            scales[:k].cpu().numpy(), opac[:k].cpu().numpy())


def _check_rows(code, ref, got, rows_src, rows_dst):
    """Compare output rows rows_dst (GPU) with rows_src of the oracle's output: bit-exact except
    the split children's means and log-scales (fp32 arithmetic against FP64)."""
    for k in PARAMS:
        a, b = ref[k][rows_src], got[k][rows_dst]
        if k in ("means", "log_scales"):
            assert np.allclose(b, a, rtol=2e-6, atol=2e-6), k
        else:
            assert np.array_equal(b, a), k


CFGS = [od.DensityConfig(split_scale=0.03),
        od.DensityConfig(split_scale=0.03, max_world_scale=0.3, max_screen_radius=20.0)]


@pytest.mark.parametrize("n,seed", [(20_000, 1), (257, 2), (1, 3), (255, 4)])
@pytest.mark.parametrize("ci", [0, 1])
def test_densify_matches_the_oracle(n, seed, ci):
    """Element by element against the oracle: a ragged last chunk, a single Gaussian, one chunk
    minus one; without and with the size-based pruning."""
    cfg = CFGS[ci]
    state = S.density_state(seed, n)
    f, m, v, acc, cnt, mr, z = state
    code, ref, rm, rv = od.densify(f, m, v, acc, cnt, mr, z, cfg)
    out, om, ov, count, flags, stats, scales, opac = _gpu_densify(state, cfg)
    assert flags == 0
    assert count == od.output_count(code)
    rows = np.arange(count)
    _check_rows(code, ref, out, rows, rows)
    src = np.repeat(np.arange(n), [od.OUTPUTS[int(c)] for c in code])
    copied = code[src] != od.SPLIT
    for k in ("means", "log_scales"):   # exact where no arithmetic happens
        assert np.array_equal(out[k][copied], ref[k][copied]), k
    for d_ref, d_got in ((rm, om), (rv, ov)):
        for k in PARAMS:
            assert np.array_equal(d_got[k], d_ref[k]), k
    for s in stats:
        assert not s.any()
    assert np.allclose(scales, np.exp(ref["log_scales"]), rtol=3e-6)
    assert np.allclose(opac, 1 / (1 + np.exp(-ref["logit_opacities"])), rtol=3e-6, atol=1e-7)


def test_densify_many_chunks_sampled():
    """1M Gaussians (3907 chunks, the look-back across many predecessors): the count exactly and
    2000 sampled sources row by row against the oracle run on those sources alone."""
    n = 1_000_000
    cfg = CFGS[1]
    state = S.density_state(11, n)
    f, m, v, acc, cnt, mr, z = state
    code = od.decide(f["logit_opacities"], f["log_scales"], acc, cnt, mr, cfg)
    offs = od.output_offsets(code)
    out, om, ov, count, flags, _, _, _ = _gpu_densify(state, cfg)
    assert flags == 0 and count == od.output_count(code)
    rng = np.random.default_rng(12)
    pick = np.sort(rng.choice(n, 2000, replace=False))
    pick = pick[code[pick] != od.PRUNE]
    sub = lambda d: {k: d[k][pick] for k in PARAMS}
    c2, ref, rm, rv = od.densify(sub(f), sub(m), sub(v), acc[pick], cnt[pick], mr[pick], z[pick], cfg)
    assert np.array_equal(c2, code[pick])
    ref_rows = od.output_offsets(c2)
    for j, i in enumerate(pick):
        k = od.OUTPUTS[int(code[i])]
        _check_rows(code, ref, out, np.arange(ref_rows[j], ref_rows[j] + k), np.arange(offs[i], offs[i] + k))
        for kk in PARAMS:
            assert np.array_equal(om[kk][offs[i]:offs[i] + k], rm[kk][ref_rows[j]:ref_rows[j] + k])
            assert np.array_equal(ov[kk][offs[i]:offs[i] + k], rv[kk][ref_rows[j]:ref_rows[j] + k])


def test_densify_capacity_overflow_writes_nothing_past_capacity():
    import torch
    n = 3000
    cfg = CFGS[0]
    state = S.density_state(5, n)
    f, m, v, acc, cnt, mr, z = state
    code, ref, _, _ = od.densify(f, m, v, acc, cnt, mr, z, cfg)
    need = od.output_count(code)
    cap = need - 777
    out, _, _, count, flags, _, _, _ = _gpu_densify(state, cfg, capacity=cap)
    assert count == need and flags & 1
    rows = np.arange(cap)
    _check_rows(code, ref, out, rows, rows)


def test_densify_empty_and_all_pruned():
    state = S.density_state(6, 0)
    *_, count, flags, _, _, _ = _gpu_densify(state, CFGS[0])
    assert count == 0 and flags == 0
    f, m, v, acc, cnt, mr, z = S.density_state(7, 1000)
    f["logit_opacities"][:] = -30.0
    *_, count, flags, _, _, _ = _gpu_densify((f, m, v, acc, cnt, mr, z), CFGS[0])
    assert count == 0 and flags == 0


def test_density_stats_of_rendered_views_match_the_oracle():
    """Two rendered views of one scene: the accumulated NDC gradient norms, counts and largest
    radii against the oracle's statistics of the same radii and gradients."""
    import torch
    from paper_2308_04079_gb300.rasterizer import Frame, GaussianTensors
    from paper_2308_04079_gb300 import _abi
    g, cam0 = S.tiny_scene(21, n=2000, width=203, height=117, deg=3)
    cams = [cam0, S.orbit_camera(3.0, 0.7, 0.2, 160, 96, 60.0)]
    gt = GaussianTensors.from_numpy(g)
    n = g.means.shape[0]
    acc = torch.zeros(n, device="cuda")
    cnt = torch.zeros(n, device="cuda")
    mr = torch.zeros(n, device="cuda")
    r_acc, r_cnt, r_mr = np.zeros(n), np.zeros(n), np.zeros(n)
    for vi, cam in enumerate(cams):
        fr = Frame(n, cam)
        fr.ensure_binned(gt)
        img, T, last = fr.outputs()
        fr.render_forward((0, 0, 0), img, T, last)
        dl = _cuda(S.upstream_grad(300 + vi, cam.height, cam.width))
        grads = fr.new_grads(gt, with_mean2d=True)
        fr.render_backward(gt, (0, 0, 0), dl, T, last, grads)
        _abi.gs_density_stats(fr.frame, grads["mean2d"].data_ptr(), acc.data_ptr(), cnt.data_ptr(), mr.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        radius = fr.view("radius", torch.int32, n).cpu().numpy()
        r_acc, r_cnt, r_mr = od.stats(grads["mean2d"].cpu().numpy(), radius, cam.width, cam.height, r_acc, r_cnt,
                                      r_mr)
    assert (r_cnt > 0).sum() > 500
    assert np.array_equal(cnt.cpu().numpy(), r_cnt)
    assert np.array_equal(mr.cpu().numpy(), r_mr)
    assert np.allclose(acc.cpu().numpy(), r_acc, rtol=2e-6, atol=1e-12)


def test_opacity_reset_matches_the_oracle():
    import torch
    from paper_2308_04079_gb300 import _abi
    rng = np.random.default_rng(8)
    n = 100_001
    raw = rng.normal(-3, 3, n).astype(np.float32)
    t, tm, tv, to = _cuda(raw), _cuda(rng.normal(size=n)), _cuda(rng.random(n)), torch.empty(n, device="cuda")
    _abi.gs_opacity_reset(t.data_ptr(), tm.data_ptr(), tv.data_ptr(), to.data_ptr(), n, 0.01,
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    want, _, _ = od.reset_opacity(raw, 0.01)
    assert np.array_equal(t.cpu().numpy().astype(np.float64), want)
    assert not tm.cpu().numpy().any() and not tv.cpu().numpy().any()
    assert np.allclose(to.cpu().numpy(), 1 / (1 + np.exp(-want)), rtol=3e-6, atol=1e-8)


def test_training_with_refinement():
    """Trainer iterations with a refinement after every step and an opacity reset every third:
    the model's tensors, moments, activated copies and statistics stay consistent in length and
    value, the Gaussian count changes, and the loss stays finite."""
    import torch
    from paper_2308_04079_gb300.density import DensityControl, DensitySchedule
    from paper_2308_04079_gb300.training import GaussianModel, Trainer
    g, cam = S.tiny_scene(31, n=3000, width=160, height=120, deg=3, log_scale_mean=-3.0)
    model = GaussianModel.from_numpy(g)
    dc = DensityControl(model, extent=2.0, grad_threshold=2e-5,
                        schedule=DensitySchedule(start=0, every=1, stop=100, reset_every=3))
    tr = Trainer(model, density=dc)
    target = _cuda(np.random.default_rng(9).random((3, cam.height, cam.width)))
    counts = [model.n]
    for it in range(6):
        before = (model.logit_opacities.cpu().numpy(), model.log_scales.cpu().numpy())
        out = tr.step(cam, target)
        torch.cuda.synchronize()
        assert np.isfinite(out.cpu().numpy()).all()
        counts.append(model.n)
        for k in PARAMS:
            assert getattr(model, k).shape[0] == model.n
            assert model.moments[k][0].shape[0] == model.n and model.moments[k][1].shape[0] == model.n
        assert model.scales.shape[0] == model.n and model.opacities.shape[0] == model.n
        assert dc.grad_accum.shape[0] == model.n and not dc.grad_accum.cpu().numpy().any()
        assert np.allclose(model.scales.cpu().numpy(), np.exp(model.log_scales.cpu().numpy()), rtol=3e-6)
    assert len(set(counts)) > 2
