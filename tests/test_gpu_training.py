"""Training step kernels against the FP64 oracle: the L1 + D-SSIM loss and its image gradient
(gs_loss_l1_dssim), the fused activation + Adam update (gs_adam_step), and one whole training
iteration on a small scene (render, loss, backward, Adam) against the oracle's iteration."""
import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import training as OT

pytestmark = pytest.mark.gpu


def _gpu_loss(x, y, lam):
    import torch
    from paper_2308_04079_gb300.training import Loss
    H, W = x.shape[1:]
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    yt = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
    d = torch.empty_like(xt)
    out = Loss(W, H, lam)(xt, yt, d)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("H,W,seed", [(37, 61, 1), (64, 64, 2), (270, 480, 3), (1, 40, 4), (33, 1, 5)])
def test_loss_and_gradient_match_the_oracle(H, W, seed):
    """Ragged sizes across the 32x32 tiles, a single row and a single column."""
    rng = np.random.default_rng(seed)
    x = rng.random((3, H, W)).astype(np.float32).astype(np.float64)
    y = np.clip(x + 0.15 * rng.standard_normal((3, H, W)), 0, 1).astype(np.float32).astype(np.float64)
    L, l1, ssim, g = OT.loss(x, y, 0.2)
    out, d = _gpu_loss(x, y, 0.2)
    assert abs(out[0] - L) <= 2e-6 and abs(out[1] - l1) <= 2e-6 and abs(out[2] - ssim) <= 2e-6, (out, L, l1, ssim)
    # the L1 part is exact up to the 1/N scale; compare the whole gradient per element against
    # its scale and per tensor in relative L2
    scale = np.abs(g).max()
    assert np.abs(d - g).max() <= 2e-3 * scale
    assert np.linalg.norm(d - g) <= 1e-4 * np.linalg.norm(g)


def test_loss_of_identical_images_is_zero():
    rng = np.random.default_rng(6)
    x = rng.random((3, 50, 70)).astype(np.float32).astype(np.float64)
    out, d = _gpu_loss(x, x, 0.2)
    assert abs(out[0]) <= 1e-6 and out[1] == 0 and abs(out[2] - 1) <= 1e-6
    assert np.abs(d).max() <= 1e-9


@pytest.mark.parametrize("act", ["none", "exp", "sigmoid"])
def test_adam_matches_the_oracle(act):
    import torch
    from paper_2308_04079_gb300 import _abi
    rng = np.random.default_rng(10)
    n = 100_003
    p = rng.standard_normal(n).astype(np.float32)
    m = (0.01 * rng.standard_normal(n)).astype(np.float32)
    v = (1e-4 * rng.random(n)).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    lr, step = 0.01, 7
    codes = {"none": _abi.GS_ACT_NONE, "exp": _abi.GS_ACT_EXP, "sigmoid": _abi.GS_ACT_SIGMOID}
    tp, tm, tv, tg = (torch.from_numpy(a.copy()).cuda() for a in (p, m, v, g))
    ta = torch.empty_like(tp)
    grp = _abi.gs_adam_group()
    grp.param, grp.grad, grp.m, grp.v, grp.activated = tp.data_ptr(), tg.data_ptr(), tm.data_ptr(), tv.data_ptr(), \
        ta.data_ptr()
    grp.n, grp.lr, grp.activation = n, lr, codes[act]
    _abi.gs_adam_step([grp], 0.9, 0.999, 1e-15, step, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    # the kernel receives its hyper-parameters as fp32: the oracle takes the same values
    b1, b2, lr32 = (float(np.float32(x)) for x in (0.9, 0.999, lr))
    p1, m1, v1, a1 = OT.adam_step(p, g, m, v, lr32, step, act, b1=b1, b2=b2, eps=float(np.float32(1e-15)))
    assert np.allclose(tm.cpu().numpy(), m1, rtol=1e-5, atol=1e-8)
    assert np.allclose(tv.cpu().numpy(), v1, rtol=1e-5, atol=1e-10)
    # the update divides by sqrt(v): compare the step itself, relative to its size
    step_gpu = p.astype(np.float64) - tp.cpu().numpy()
    step_ref = p.astype(np.float64) - p1
    assert np.all(np.abs(step_gpu - step_ref) <= 1e-4 * np.abs(step_ref) + 2e-7 * (1 + np.abs(p)))
    assert np.allclose(ta.cpu().numpy(), a1, rtol=1e-5, atol=1e-6)


def test_training_iteration_matches_the_oracle():
    """One iteration on a small scene: the raw parameters after the GPU step against the oracle's
    FP64 render, backward, loss gradient and Adam step (the first Adam step moves every
    parameter by about lr sign(g), so the comparison is on the gradients' signs and sizes)."""
    import torch
    from paper_2308_04079_gb300.training import GaussianModel, Trainer
    g, cam = S.tiny_scene(41, n=300, width=96, height=64, deg=3)
    rng = np.random.default_rng(42)
    target = rng.random((3, cam.height, cam.width)).astype(np.float32)
    model = GaussianModel.from_numpy(g)
    before = {k: getattr(model, k).cpu().numpy().astype(np.float64)
              for k in ("means", "log_scales", "quats", "logit_opacities", "sh")}
    tr = Trainer(model, eps=1e-15)
    out = tr.step(cam, torch.from_numpy(target).cuda())
    torch.cuda.synchronize()
    # oracle: forward, loss gradient, backward, Adam (step 1)
    orc = oracle.render_forward(g, cam, (0, 0, 0))
    L, _, _, dimg = OT.loss(orc["img"], target, 0.2)
    assert abs(float(out[0].item()) - L) <= 1e-4 * max(1.0, L)
    ob = oracle.render_backward(g, cam, dimg, (0, 0, 0))
    # The comparison is of Adam steps, whose sign follows the gradient's: an element whose
    # gradient the oracle's allowance (decisions near their threshold, flipped) could move by
    # a tenth of its size or more is left out of the sign check, every other one is in it.
    touched = np.abs(ob["opacities"]) > 0
    grad_of = {"means": "means", "log_scales": "scales", "quats": "quats", "logit_opacities": "opacities"}
    lr = tr.lr
    ref = {
        "means": OT.adam_step(before["means"], ob["means"], 0, 0, lr["means"], 1)[0],
        "log_scales": OT.adam_step(before["log_scales"], ob["scales"], 0, 0, lr["log_scales"], 1, "exp")[0],
        "quats": OT.adam_step(before["quats"], ob["quats"], 0, 0, lr["quats"], 1)[0],
        "logit_opacities": OT.adam_step(before["logit_opacities"], ob["opacities"], 0, 0,
                                        lr["logit_opacities"], 1, "sigmoid")[0],
    }
    for k, r in ref.items():
        got = getattr(model, k).cpu().numpy().astype(np.float64)
        gstar = np.abs(ob[grad_of[k]])
        sure = (np.asarray(ob["allow"][grad_of[k]]) < 0.1 * gstar)
        sure = (sure & touched.reshape((-1,) + (1,) * (gstar.ndim - 1))).reshape(-1)
        assert sure.mean() > 0.5
        dg, dr = (got - before[k]).reshape(-1), (r - before[k]).reshape(-1)
        # a first Adam step is +-lr wherever |g| >> eps: the signs must agree where the oracle's
        # gradient is clearly non-zero, and the sizes everywhere
        big = (np.abs(dr) > 0.5 * lr[k]) & sure
        agree = np.mean(np.sign(dg[big]) == np.sign(dr[big]))
        assert agree >= 0.995, (k, agree)
        assert np.all(np.abs(dg) <= lr[k] * (1 + 1e-4) + 1e-7), k


def test_sh_band_schedule_moves_only_the_active_bands():
    """Sec. 7.1: zero-order band first, one more band every sh_band_every iterations; the
    rasterizer zeroes the gradients of the unused coefficients, so Adam leaves them alone."""
    import torch
    from paper_2308_04079_gb300.training import GaussianModel, Trainer
    g, cam = S.tiny_scene(51, n=400, width=80, height=60, deg=3)
    model = GaussianModel.from_numpy(g)
    tr = Trainer(model, sh_band_every=2)
    target = torch.from_numpy(np.random.default_rng(52).random((3, cam.height, cam.width), dtype=np.float32)).cuda()
    sh0 = model.sh.cpu().numpy().copy()
    tr.step(cam, target)                       # iteration 0: degree 0
    torch.cuda.synchronize()
    sh1 = model.sh.cpu().numpy()
    assert np.abs(sh1[:, 0] - sh0[:, 0]).max() > 0
    assert np.array_equal(sh1[:, 1:], sh0[:, 1:])
    tr.step(cam, target)                       # iteration 1: degree 0
    tr.step(cam, target)                       # iteration 2: degree 1
    torch.cuda.synchronize()
    sh3 = model.sh.cpu().numpy()
    assert np.abs(sh3[:, 1:4] - sh0[:, 1:4]).max() > 0
    assert np.array_equal(sh3[:, 4:], sh0[:, 4:])
