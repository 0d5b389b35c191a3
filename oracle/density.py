"""FP64 oracle of the adaptive density control of Sec. 5.2 (Algorithm 1, the refinement step):
view-space gradient statistics, pruning, cloning, splitting and the opacity reset.

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the CPU legs of bench.py use this
module; it shares no code with the CUDA path and the product path never calls it.

Readings (the paper gives tau_pos = 0.0002, phi = 1.6, the 100-iteration densification period
and the 3000-iteration opacity reset; everything else below is a reading):
  * view-space positional gradient = gradient of the loss with respect to the projected mean
    in normalised device coordinates (u_ndc = 2 u / W - 1), i.e. the pixel gradient scaled by
    (W / 2, H / 2); its magnitude is averaged over the views in which the Gaussian was not
    culled (screen radius > 0);
  * "||S|| > tau_S" compares the largest scale component; "IsTooLarge" is the largest scale
    component above a world-space limit or the largest screen radius seen since the last
    refinement above a pixel limit (each limit optional);
  * every comparison is strict, as Algorithm 1 writes them: prune when alpha < epsilon_alpha,
    densify when the mean gradient > tau_pos, split when the scale > tau_S;
  * pruning wins: a pruned Gaussian is neither cloned nor split;
  * clone = an exact copy placed right after the original (its later displacement along the
    positional gradient comes from the optimiser, whose moments start at zero for the copy);
  * split = two children in place of the original, each with the original's mean plus
    R(q) diag(s) z for a standard normal draw z (the original Gaussian as the sampling
    density, pre-split scale s), raw log-scale lowered by ln(phi) (scale divided by phi), the
    other attributes copied and optimiser moments zero (a zero quaternion, which the renderer
    culls in every view, splits with the identity rotation);
  * outputs keep the source order, each source's outputs adjacent;
  * decisions (integers from floating point) are taken in fp32 as the kernels take them:
    opacity against epsilon_alpha in the raw (logit) domain, scales in the raw (log) domain,
    each threshold transformed in double and rounded to fp32 once; the mean gradient as one
    fp32 division accum / count;
  * opacity reset: opacity <- min(opacity, max_opacity) (max_opacity 0.01, "close to zero"),
    compared and clamped in the raw domain against fp32(logit(max_opacity)); the optimiser
    moments of every opacity restart at zero."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import quat_to_rot

PARAMS = ("means", "log_scales", "quats", "logit_opacities", "sh")

# decision codes
PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3
OUTPUTS = {PRUNE: 0, KEEP: 1, CLONE: 2, SPLIT: 2}


@dataclass
class DensityConfig:
    grad_threshold: float = 0.0002     # tau_pos (Sec. 5.2)
    min_opacity: float = 0.005         # epsilon_alpha
    split_scale: float = 0.03          # tau_S, world units
    max_world_scale: float = 0.0       # <= 0: no world-size pruning
    max_screen_radius: float = 0.0     # <= 0: no screen-size pruning
    split_factor: float = 1.6          # phi (Sec. 5.2)


def stats(mean2d_grad, radius, width: int, height: int, accum, count, max_radius):
    """Add one view: for every Gaussian with radius > 0, accum += |(gu W/2, gv H/2)|,
    count += 1, max_radius = max(max_radius, radius).  Returns new arrays."""
    g = np.asarray(mean2d_grad, np.float64).reshape(-1, 2)
    r = np.asarray(radius).reshape(-1)
    vis = r > 0
    norm = np.hypot(g[:, 0] * (width / 2.0), g[:, 1] * (height / 2.0))
    accum = np.asarray(accum, np.float64) + np.where(vis, norm, 0.0)
    count = np.asarray(count, np.float64) + vis
    max_radius = np.where(vis, np.maximum(np.asarray(max_radius, np.float64), r), max_radius)
    return accum, count, max_radius


def raw_thresholds(cfg: DensityConfig):
    """fp32 thresholds in the raw parameter domains: logit(epsilon_alpha), ln(tau_S),
    ln(world limit), and the raw log-scale step ln(phi)."""
    eps = float(cfg.min_opacity)
    logit = np.float32(np.log(eps / (1.0 - eps)))
    ln_split = np.float32(np.log(cfg.split_scale)) if cfg.split_scale > 0 else np.float32(np.inf)
    ln_world = np.float32(np.log(cfg.max_world_scale)) if cfg.max_world_scale > 0 else np.float32(np.inf)
    return logit, ln_split, ln_world, np.float32(np.log(cfg.split_factor))


def decide(logit_opacities, log_scales, accum, count, max_radius, cfg: DensityConfig) -> np.ndarray:
    """Algorithm 1's refinement decision of every Gaussian (PRUNE, KEEP, CLONE, SPLIT), in fp32."""
    logit_thr, ln_split, ln_world, _ = raw_thresholds(cfg)
    o = np.asarray(logit_opacities, np.float32).reshape(-1)
    smax = np.asarray(log_scales, np.float32).reshape(-1, 3).max(axis=1)
    acc = np.asarray(accum, np.float32).reshape(-1)
    cnt = np.asarray(count, np.float32).reshape(-1)
    mr = np.asarray(max_radius, np.float32).reshape(-1)
    prune = o < logit_thr
    prune |= smax > ln_world
    if cfg.max_screen_radius > 0:
        prune |= mr > np.float32(cfg.max_screen_radius)
    with np.errstate(divide="ignore", invalid="ignore"):
        avg = np.where(cnt > 0, acc / np.where(cnt > 0, cnt, np.float32(1)), np.float32(0))
    dens = (cnt > 0) & (avg > np.float32(cfg.grad_threshold)) & ~prune
    code = np.full(o.shape, KEEP, np.int32)
    code[prune] = PRUNE
    code[dens & (smax > ln_split)] = SPLIT
    code[dens & ~(smax > ln_split)] = CLONE
    return code


def densify(params: dict, m: dict, v: dict, accum, count, max_radius, normals, cfg: DensityConfig):
    """One refinement step.  params / m / v map PARAMS to [n, ...] arrays (raw values and the
    Adam moments); normals is [n, 2, 3] of standard normal draws (used by split sources only).
    Returns (code, out_params, out_m, out_v) with outputs in source order."""
    n = np.asarray(params["means"]).shape[0]
    code = decide(params["logit_opacities"], params["log_scales"], accum, count, max_radius, cfg)
    ln_phi = np.log(cfg.split_factor)
    z = np.asarray(normals, np.float64).reshape(n, 2, 3) if n else np.zeros((0, 2, 3))
    P = {k: np.asarray(params[k], np.float64) for k in PARAMS}
    Pm = {k: np.asarray(m[k], np.float64) for k in PARAMS}
    Pv = {k: np.asarray(v[k], np.float64) for k in PARAMS}
    rows = {k: [] for k in PARAMS}
    rows_m = {k: [] for k in PARAMS}
    rows_v = {k: [] for k in PARAMS}
    for i in range(n):
        c = code[i]
        if c == PRUNE:
            continue
        src = {k: P[k][i] for k in PARAMS}
        sm = {k: Pm[k][i] for k in PARAMS}
        sv = {k: Pv[k][i] for k in PARAMS}
        if c == KEEP or c == CLONE:
            for k in PARAMS:
                rows[k].append(src[k])
                rows_m[k].append(sm[k])
                rows_v[k].append(sv[k])
            if c == CLONE:
                for k in PARAMS:
                    rows[k].append(src[k])
                    rows_m[k].append(np.zeros_like(sm[k]))
                    rows_v[k].append(np.zeros_like(sv[k]))
            continue
        # split: sample both children from N(mu, R diag(s)^2 R^T)
        q = src["quats"]
        qn = np.linalg.norm(q)
        R = quat_to_rot(q / qn) if qn > 0 else np.eye(3)   # the renderer's rotation R(q / |q|)
        s = np.exp(src["log_scales"])
        for child in range(2):
            for k in PARAMS:
                if k == "means":
                    val = src["means"] + R @ (s * z[i, child])
                elif k == "log_scales":
                    val = src["log_scales"] - ln_phi
                else:
                    val = src[k]
                rows[k].append(val)
                rows_m[k].append(np.zeros_like(sm[k]))
                rows_v[k].append(np.zeros_like(sv[k]))

    def stack(d):
        out = {}
        for k in PARAMS:
            shape = np.asarray(params[k]).shape[1:]
            out[k] = np.array(d[k], np.float64).reshape((-1,) + shape)
        return out
    return code, stack(rows), stack(rows_m), stack(rows_v)


def output_count(code) -> int:
    return int(sum(OUTPUTS[int(c)] for c in np.asarray(code).reshape(-1)))


def output_offsets(code) -> np.ndarray:
    """First output row of every source: the number of rows its predecessors produce."""
    counts = np.array([OUTPUTS[int(c)] for c in np.asarray(code).reshape(-1)], np.int64)
    return np.concatenate([[0], np.cumsum(counts)[:-1]]) if counts.size else counts


def reset_opacity(logit_opacities, max_opacity: float = 0.01):
    """opacity <- min(opacity, max_opacity), in the raw domain.  Returns (raw, m, v) with the
    moments zero."""
    raw = np.asarray(logit_opacities, np.float32)
    cap = np.float32(np.log(max_opacity / (1.0 - max_opacity)))
    out = np.where(raw > cap, cap, raw).astype(np.float64)
    return out, np.zeros_like(out), np.zeros_like(out)
