"""Helpers for the CUDA parity tests: run the C-ABI stages on seeded inputs and compare
with the FP64 oracle.  The oracle sees the generator's inputs; the one exception is the
binning check, which (as the binning definition is exact on given fp32 screen values) feeds
the GPU's own fp32 screen means, depths and radii to the oracle's binning and requires the
same keys, order and ranges bit for bit.

Every pixel and every Gaussian is checked.  A pixel or Gaussian that a decision near its
threshold touches (the oracle lists such decisions and evaluates each one the other way) may
match the flipped alternative instead of the definition, or, when several flip together, lie
within the definition plus the summed magnitude of the flips' effects."""
from __future__ import annotations

import numpy as np

IMG_ATOL = 1e-4          # images and final transmittance, absolute per channel (fp32 vs fp64)
GRAD_REL_L2 = 1e-3       # gradients: per-tensor relative L2 error
GRAD_ELEM_REL = 1e-3     # gradients: per element, relative to max(|g*|, GRAD_FLOOR * max|g*|)
GRAD_FLOOR = 1e-3

# one line per comparison, printed at the end of the session by conftest.py
REPORT: list[str] = []


def _assert_status_ok(fr):
    """No device-side condition but culled non-finite inputs (synchronises)."""
    from paper_2308_04079_gb300 import _abi
    code, st = fr.status()
    assert code in (_abi.GS_OK, _abi.GS_ERR_NUMERIC), (_abi.status_string(code), st.flags)


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
    _assert_status_ok(fr)
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
    _assert_status_ok(fr)
    n = gt.n
    grad2d = fr.view("grad2d", torch.float32, 12 * n).view(n, 12).clone()
    L = fr.view("conic_opacity", torch.float32, 4 * n).view(n, 4)[:, :3].clone()
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items() if v is not None}
    g2 = grad2d.cpu().numpy().astype(np.float64)
    l11, l21, l22 = (L.cpu().numpy().astype(np.float64)[:, k] for k in range(3))
    # the mean and Sigma' sums are in the whitened frame of the conic's Cholesky factor L:
    # dL/d(u, v) = L (P, Q), dL/dSigma' = L K L^T
    P, Q, K00, K01, K11 = (g2[:, k] for k in range(5))
    out["uv"] = np.stack([l11 * P, l21 * P + l22 * Q], 1)
    a00 = l11 * l11 * K00
    a01 = l11 * (l21 * K00 + l22 * K01)
    a11 = l21 * l21 * K00 + 2 * l21 * l22 * K01 + l22 * l22 * K11
    out["cov2d"] = np.stack([a00, a01, a11], 1)
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


def compare_images(gpu, orc, atol=IMG_ATOL, check_last=True, mask=None, label=""):
    """Image, T and last contributor on every pixel (of ``mask``, if given): within ``atol``
    of the oracle's definition and the same last Gaussian; where the oracle lists decisions
    near their threshold, matching one flipped alternative (image, T within ``atol``, same last
    Gaussian) also passes, and so does lying within ``atol`` plus the summed effect of the
    pixel's alternatives with the last Gaussian of the definition or of one alternative."""
    H, W = orc["T"].shape
    img_g, img_o = gpu["img"].reshape(3, -1), orc["img"].reshape(3, -1)
    T_g, T_o = gpu["T"].reshape(-1), orc["T"].reshape(-1)
    lid_g, lid_o = gpu["last_id"].reshape(-1), orc["last_id"].reshape(-1)
    sel = np.ones(H * W, bool) if mask is None else np.asarray(mask, bool).reshape(-1)
    err = np.maximum(np.abs(img_g - img_o).max(axis=0), np.abs(T_g - T_o))
    same_last = (lid_g == lid_o) | (not check_last)
    dec = orc["pix_dec"].reshape(-1) != 0
    plain = sel & ~dec
    main_ok = (err <= atol) & same_last
    alt = orc["alt"]
    ap = alt["pix"]
    use = sel[ap]
    ap = ap[use]
    a_img, a_T, a_last = alt["img"][use], alt["T"][use], alt["last_id"][use]
    a_err = np.maximum(np.abs(img_g[:, ap].T - a_img).max(axis=1), np.abs(T_g[ap] - a_T))
    a_last_ok = (lid_g[ap] == a_last) | (not check_last)
    alt_ok = np.zeros(H * W, bool)
    np.logical_or.at(alt_ok, ap, (a_err <= atol) & a_last_ok)
    effect = np.zeros(H * W)
    np.add.at(effect, ap, np.maximum(np.abs(a_img - img_o[:, ap].T).max(axis=1), np.abs(a_T - T_o[ap])))
    last_any = same_last.copy()
    np.logical_or.at(last_any, ap, a_last_ok)
    bound_ok = (err <= atol + effect) & last_any
    flagged = sel & dec
    ok = np.where(flagged, main_ok | alt_ok | bound_ok, main_ok)
    n = int(sel.sum())
    stats = dict(pixels=n, flagged_frac=float(flagged.sum()) / max(n, 1),
                 max_err_plain=float(err[plain].max(initial=0.0)),
                 flagged_match_definition=int((flagged & main_ok).sum()),
                 flagged_match_alternative=int((flagged & ~main_ok & alt_ok).sum()),
                 flagged_within_bound=int((flagged & ~main_ok & ~alt_ok & bound_ok).sum()),
                 failed=int((sel & ~ok).sum()), dec_overflow=orc.get("dec_overflow", 0))
    REPORT.append(f"image {label}: {n} px, flagged {stats['flagged_frac']:.4%} "
                  f"(= definition {stats['flagged_match_definition']}, = alternative "
                  f"{stats['flagged_match_alternative']}, within bound {stats['flagged_within_bound']}), "
                  f"max error elsewhere {stats['max_err_plain']:.2e}, failed {stats['failed']}")
    assert stats["dec_overflow"] == 0, stats
    assert stats["failed"] == 0, (stats, np.nonzero(sel & ~ok)[0][:10])
    return stats


def compare_grads(gpu, orc, names=("means", "scales", "quats", "opacities", "sh"), rel=GRAD_REL_L2,
                  elem_rel=GRAD_ELEM_REL, floor=GRAD_FLOOR, label="", select=None):
    """Every Gaussian (of ``select``, if given): per element |g - g*| <= elem_rel *
    max(|g*|, floor * max|g*|) + a, with a the oracle's allowance (the summed magnitude of the
    changes that the decisions near their threshold make when flipped; 0 for a Gaussian that no
    such decision touches); per tensor ||g - g*|| <= rel ||g*|| + ||a||.  A Gaussian with no
    oracle gradient and no allowance must get exactly zero."""
    allow = orc["allow"]
    cond = orc.get("cond", {})
    stats = {}
    parts = []
    for name in names:
        b = np.asarray(orc[name])
        n = b.shape[0]
        b = b.reshape(n, -1)
        a = np.asarray(gpu[name]).reshape(n, -1)[:, : b.shape[1]]
        A = np.asarray(allow[name]).reshape(n, -1)[:, : b.shape[1]]
        Cn = np.asarray(cond[name]).reshape(n, -1)[:, : b.shape[1]] if name in cond else np.zeros_like(A)
        sel = np.ones(n, bool) if select is None else np.asarray(select, bool)
        a, b, A, Cn = a[sel], b[sel], A[sel], Cn[sel]
        mx = float(np.abs(b).max(initial=0.0))
        tol = elem_rel * np.maximum(np.abs(b), floor * mx)
        d = np.abs(a - b)
        bad = d > tol + A + Cn
        used = (d > tol) & ~bad
        used_cond = (d > tol + A) & ~bad
        A = A + Cn
        zero = (b == 0) & (A == 0)
        nz = int((zero & (a != 0)).sum())
        l2 = float(np.linalg.norm(a - b))
        l2_lim = rel * float(np.linalg.norm(b)) + float(np.linalg.norm(A))
        worst = float((d / np.maximum(tol + A, 1e-300)).max(initial=0.0))
        stats[name] = dict(elements=int(b.size), rel_l2=l2 / max(float(np.linalg.norm(b)), 1e-300),
                           worst_frac_of_bound=worst, with_allowance=int((A.max(axis=1) > 0).sum()),
                           needed_allowance=int(used.sum()), needed_conditioning=int(used_cond.sum()),
                           failed=int(bad.sum()), nonzero_untouched=nz)
        parts.append(f"{name} {stats[name]['rel_l2']:.1e}/{worst:.2f}/{int(used.sum())}/{int(used_cond.sum())}")
        assert not bad.any(), (name, stats[name], np.argwhere(bad)[:5])
        assert l2 <= l2_lim, (name, stats[name])
        assert nz == 0, (name, stats[name])
    w = int((np.asarray(allow["opacities"]).reshape(-1) > 0).sum())
    REPORT.append(f"grads {label}: Gaussians with a decision allowance {w}; per tensor rel-L2/worst element "
                  f"as a fraction of its bound/elements beyond 1e-3 max(|g*|, 1e-3 max|g*|) (within the "
                  f"allowances)/of those, beyond the decision allowance (within the fp32 conditioning "
                  f"allowance): " + ", ".join(parts))
    return stats


def oracle_view_sum(g, cams, dimgs, bg, cfg=None, masks=None,
                    names=("means", "scales", "quats", "opacities", "sh")):
    """The oracle's gradients summed over several views of one scene, with the allowances of
    every view summed alike."""
    import oracle
    total, allow = None, None
    for v, cam in enumerate(cams):
        ob = oracle.render_backward(g, cam, dimgs[v], bg, cfg, tile_mask=None if masks is None else masks[v])
        assert ob["dec_overflow"] == 0
        if total is None:
            total = {k: ob[k].copy() for k in names}
            allow = {k: ob["allow"][k].copy() for k in names}
            cond = {k: ob["cond"][k].copy() for k in names}
        else:
            for k in names:
                total[k] += ob[k]
                allow[k] += ob["allow"][k]
                cond[k] += ob["cond"][k]
    total["allow"] = allow
    total["cond"] = cond
    return total
