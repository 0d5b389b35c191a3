"""Helpers for the CUDA parity tests: run the C-ABI stages on seeded inputs and compare
with the FP64 oracle.  The oracle only ever sees the generator's inputs; nothing computed
by the CUDA path is fed to it."""
from __future__ import annotations

import numpy as np

# Tolerances, from the fp32 arithmetic of the kernels against the FP64 oracle: pixels and
# Gaussians with a decision near its threshold (the oracle's ambiguity flags) are excluded.
IMG_ATOL = 1e-4          # images and final transmittance, absolute per channel (fp32 vs fp64)
GRAD_REL_L2 = 1e-3       # gradients: per-tensor relative L2 error
GRAD_ELEM_REL = 1e-2     # gradients: per element, relative to max(|g*|, rms of the tensor)


def gpu_frame(g_np, cam, cfg=None, capacity=None):
    import torch
    from paper_2308_04079_gb300 import Frame, GaussianTensors
    gt = GaussianTensors.from_numpy(g_np).prepared()
    fr = Frame(gt.n, cam, cfg, capacity=capacity)
    return fr, gt


def gpu_forward(g_np, cam, bg, cfg=None, capacity=None):
    """preprocess + bin_sort + render_forward through the C ABI; returns numpy outputs."""
    import torch
    fr, gt = gpu_frame(g_np, cam, cfg, capacity)
    fr.ensure_binned(gt)
    img, T, last = fr.outputs()
    fr.render_forward(bg, img, T, last)
    torch.cuda.synchronize()
    last_np = last.cpu().numpy()
    return dict(img=img.cpu().numpy().astype(np.float64), T=T.cpu().numpy().astype(np.float64),
                last=last_np, last_id=last_contributor_ids(fr, last_np), frame=fr, g=gt, img_t=img, T_t=T,
                last_t=last)


def last_contributor_ids(fr, last):
    """Gaussian index of every pixel's last contributor (-1 = none): the GPU's `last` is a
    1-based position in its tile's instance list, the oracle's list may hold other (never
    blended) splats, so the two are compared by Gaussian index."""
    import torch
    _, st = fr.status()
    K = min(int(st.num_instances), fr.capacity)
    ranges = fr.view("ranges", torch.int32, 2 * fr.tiles).view(-1, 2).cpu().numpy().astype(np.int64)
    vals = fr.view("vals_sorted", torch.int32, max(K, 1)).cpu().numpy().astype(np.int64)
    H, W = last.shape
    tw, th = fr.cfg.tile_w, fr.cfg.tile_h
    TX = (W + tw - 1) // tw
    py, px = np.mgrid[0:H, 0:W]
    t = (py // th) * TX + px // tw
    pos = ranges[t, 0] + last.astype(np.int64) - 1
    out = np.full(last.shape, -1, np.int64)
    hit = last > 0
    out[hit] = vals[pos[hit]]
    return out


def gpu_backward(run, bg, dimg_np):
    import torch
    fr, gt = run["frame"], run["g"]
    grads = fr.new_grads(gt)
    d = torch.from_numpy(np.ascontiguousarray(dimg_np, dtype=np.float32)).cuda()
    fr.render_backward(gt, bg, d, run["T_t"], run["last_t"], grads)
    n = gt.n
    grad2d = fr.view("grad2d", torch.float32, 12 * n).view(n, 12).clone()
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items() if v is not None}
    g2 = grad2d.cpu().numpy().astype(np.float64)
    out["uv"] = g2[:, 0:2]
    out["cov2d"] = g2[:, 2:5]
    out["opac2d"] = g2[:, 5]
    out["rgb"] = g2[:, 6:9]
    return out


def screen_state(run):
    """Per-Gaussian screen-space outputs of gs_preprocess read from the workspace."""
    import torch
    fr, n = run["frame"], run["g"].n
    xy4 = fr.view("xy", torch.float32, 4 * n).view(n, 4).cpu().numpy().astype(np.float64)
    xy = xy4[:, 0:2] + xy4[:, 2:4]                      # double-float (hi + lo)
    depth = fr.view("depth", torch.float32, n).cpu().numpy()
    co = fr.view("conic_opacity", torch.float32, 4 * n).view(n, 4).cpu().numpy()
    L = co[:, :3].astype(np.float64)                    # Cholesky factor of the conic
    conic = np.stack([L[:, 0] ** 2, L[:, 0] * L[:, 1], L[:, 1] ** 2 + L[:, 2] ** 2], 1)
    rgb = fr.view("rgb", torch.float32, 4 * n).view(n, 4).cpu().numpy()
    radius = fr.view("radius", torch.int32, n).cpu().numpy()
    return dict(xy=xy, xy_hi=xy4[:, 0:2], depth=depth, conic=conic, opacity=co[:, 3], rgb=rgb[:, :3],
                radius=radius)


def compare_images(gpu, orc, max_amb_frac=0.01, atol=IMG_ATOL, check_last=True):
    """Element-wise image / T / last comparison on pixels without an ambiguous decision."""
    amb = (orc["pix_amb"] & 1) != 0
    frac = float(amb.mean())
    ok = ~amb
    err_img = np.abs(gpu["img"] - orc["img"]).max(axis=0)
    err_T = np.abs(gpu["T"] - orc["T"])
    stats = dict(amb_frac=frac, max_img_err=float(err_img[ok].max(initial=0.0)),
                 max_T_err=float(err_T[ok].max(initial=0.0)), pixels=int(ok.sum()))
    assert frac <= max_amb_frac, stats
    assert stats["max_img_err"] <= atol, stats
    assert stats["max_T_err"] <= atol, stats
    if check_last:
        sure = (orc["pix_amb"] & 5) == 0            # no decision near any threshold
        mism = (gpu["last_id"] != orc["last_id"]) & sure
        stats["last_mismatch"] = int(mism.sum())
        assert stats["last_mismatch"] == 0, stats
    return stats


def compare_grads(gpu, orc, keep, names=("means", "scales", "quats", "opacities", "sh"), rel=GRAD_REL_L2,
                  elem_rel=GRAD_ELEM_REL):
    """Per-tensor relative L2 error <= rel over the Gaussians in ``keep``, and per element
    |g - g*| <= elem_rel * max(|g*|, rms(g*)) (fp32 sums of many signed terms)."""
    stats = {}
    for name in names:
        a = gpu[name][keep].reshape(keep.sum(), -1)
        b = orc[name][keep].reshape(keep.sum(), -1)
        if name == "sh":
            a = a[:, : b.shape[1]]
        nb = np.linalg.norm(b)
        err = np.linalg.norm(a - b) / max(nb, 1e-30)
        rms = float(np.sqrt(np.mean(b ** 2))) if b.size else 0.0
        scale = np.maximum(np.abs(b), rms)
        elem = float((np.abs(a - b) / np.maximum(scale, 1e-30)).max(initial=0.0))
        stats[name] = (float(err), elem)
        assert err <= rel, (name, stats)
        assert elem <= elem_rel, (name, stats)
    return stats
