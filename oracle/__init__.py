"""FP64 CPU oracle of the 3D Gaussian Splatting tile rasterizer (Kerbl et al. 2023).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
It shares no code with the CUDA path (``paper_2308_04079_gb300``) and never imports it;
the product path never imports this package.

Functions (each a thin ctypes marshaller around ``gs_oracle.c``):

* :func:`preprocess`       per-Gaussian cull / EWA projection / radius / tile rectangle /
                           SH colour (Sec. 4, Sec. 6, eq. volume-render, eq. quat).
* :func:`bin_instances`    the binning definition of App. C / Algorithm 2 on given fp32
                           screen-space values: keys, one stable sort, tile ranges.
* :func:`render_forward`   per-pixel front-to-back blending, eq. front-to-back, with the
                           App. C numerical-stability rules.
* :func:`render_backward`  analytic FP64 gradients (Sec. 6 traversal, App. A chain rule).
* :func:`sh_eval`          real spherical-harmonic basis, bands 0..3, and its gradient.
* :func:`quat_to_rot`      eq. quat of App. A.
* :func:`render_forward_isotropic`, :func:`render_backward_isotropic`  the isotropic ablation
                           of Sec. 7.3 (one scale per Gaussian) through the definitions above.

The Limited-BW ablation of Sec. 7.3 is ``cfg_array(grad_limit=N)``: gradients reach only the
N front-most blended Gaussians of each pixel.

Every discrete decision (cull, radius, tile rectangle, skip, clamp, stop, depth order) that
lies within the error margin of an FP32 evaluation of its threshold is reported, and each is
evaluated the other way too: :func:`render_forward` returns the flipped alternatives of every
such pixel (``alt``), :func:`render_backward` the per-Gaussian sum of the magnitudes of the
changes they make to the gradients (``allow``).  Tests check every pixel and every Gaussian
against them instead of excluding any.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# per-Gaussian bits of the per-Gaussian stage (preprocess)
AMB_CULL = 1
AMB_RECT = 2
AMB_RGB = 4
# kinds of pixel decision near a threshold; pix_dec has bit (kind - 1) set for each kind present
DEC_SKIP = 1    # alpha < 1/255 (App. C)
DEC_CLAMP = 2   # alpha clamped at 0.99 (App. C)
DEC_STOP = 3    # stop before T (1 - alpha) < 1e-4 (App. C)
DEC_SWAP = 4    # equal or adjacent fp32 depth keys
DEC_DROP = 5    # tile membership near its threshold: the Gaussian may be absent
DEC_ADD = 6     # a Gaussian outside the tile's list may be in it

U = 2.0 ** -24  # unit roundoff of IEEE fp32

DEFAULT_CFG = dict(
    tile_w=16, tile_h=16,          # Sec. 6 / App. C: 16x16 tiles
    alpha_min=1.0 / 255.0,         # App. C: skip alpha < 1/255
    alpha_max=0.99,                # App. C: clamp alpha at 0.99
    T_min=1e-4,                    # App. C: stop before accumulated opacity exceeds 0.9999
    dilation=0.3,                  # low-pass filter added to the diagonal of Sigma'
    guard=1.3,                     # guard band on the frustum tangents (Sec. 6)
    extent=3.0,                    # 3-sigma screen extent (Sec. 6, 99% interval)
    radius_max=1 << 24,            # radius clamp (pixels)
    eps_geom=2e-6,                 # margin, geometric decisions (relative): ~32 u
    eps_alpha=3e-5,                # margin, o G at the skip / clamp thresholds (relative), besides the power's
    eps_T=1e-3,                    # margin, transmittance at the stop threshold (relative)
    grad_limit=0,                  # > 0: gradients for the N front-most blended Gaussians only
    eps_power=20 * U,              # margin of the power relative to its terms' magnitude sum (gs_oracle.c)
)

_lib = None


def _load():
    global _lib
    if _lib is None:
        # GS_ORACLE_LIB: a differently built oracle library (the mutant tests plant errors in a
        # copy of gs_oracle.c and check that the pins catch them)
        path = os.environ.get("GS_ORACLE_LIB") or _build.build()
        lib = ctypes.CDLL(path)
        D = ctypes.POINTER(ctypes.c_double)
        I32 = ctypes.POINTER(ctypes.c_int32)
        U32 = ctypes.POINTER(ctypes.c_uint32)
        U8 = ctypes.POINTER(ctypes.c_uint8)
        F = ctypes.POINTER(ctypes.c_float)
        U64 = ctypes.POINTER(ctypes.c_uint64)
        L = ctypes.c_long
        lib.orc_quat_to_rot.argtypes = [D, D]
        lib.orc_sh_eval.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D]
        lib.orc_preprocess.argtypes = [L, D, D, D, D, D, ctypes.c_int, ctypes.c_int, D, D,
                                       I32, D, D, D, D, I32, I32, D, D, U32, I32, I32]
        I64 = ctypes.POINTER(ctypes.c_int64)
        LP = ctypes.POINTER(ctypes.c_long)
        lib.orc_render_forward.argtypes = [L, D, D, D, D, D, ctypes.c_int, ctypes.c_int, D, D,
                                           D, U8, D, D, I32, I32, U8, U32, L, I64, I32, D, D, I32, LP]
        lib.orc_render_backward.argtypes = [L, D, D, D, D, D, ctypes.c_int, ctypes.c_int, D, D,
                                            D, U8, D, D, D, D, D, D, D, D, D, D, U8, U32,
                                            D, D, D, D, D, D, D, D, D, D, LP]
        lib.orc_bin.argtypes = [L, F, F, I32, F, F, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                L, U64, U32, U32]
        lib.orc_bin.restype = L
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_reach_needed.argtypes = [L, D, D, D, D, D, ctypes.c_int, ctypes.c_int, D, D, L, I64]
        lib.orc_reach_needed.restype = L
        _lib = lib
    return _lib


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def cam_array(cam) -> np.ndarray:
    """Flatten a camera (width, height, fx, fy, cx, cy, R (world->camera), t, near)."""
    a = np.zeros(19, dtype=np.float64)
    a[0], a[1] = cam.width, cam.height
    a[2], a[3], a[4], a[5] = cam.fx, cam.fy, cam.cx, cam.cy
    a[6:15] = np.asarray(cam.R, dtype=np.float64).reshape(9)
    a[15:18] = np.asarray(cam.t, dtype=np.float64).reshape(3)
    a[18] = cam.near
    return a


def cfg_array(**overrides) -> np.ndarray:
    c = dict(DEFAULT_CFG)
    for k, v in overrides.items():
        if k not in c:
            raise KeyError(k)
        c[k] = v
    return np.array([c["tile_w"], c["tile_h"], c["alpha_min"], c["alpha_max"], c["T_min"],
                     c["dilation"], c["guard"], c["extent"], c["radius_max"], c["eps_geom"],
                     c["eps_alpha"], c["eps_T"], c["grad_limit"], c["eps_power"]],
                    dtype=np.float64)


def _gauss_args(g):
    n = int(np.asarray(g.means).shape[0])
    means = _f64(g.means).reshape(n, 3)
    scales = _f64(g.scales).reshape(n, 3)
    quats = _f64(g.quats).reshape(n, 4)
    opac = _f64(g.opacities).reshape(n)
    sh = _f64(g.sh)
    sh_stride = sh.shape[1]
    return n, means, scales, quats, opac, sh, int(g.sh_degree), int(sh_stride)


def tiles_xy(cam, cfg: np.ndarray):
    tw, th = int(cfg[0]), int(cfg[1])
    return (cam.width + tw - 1) // tw, (cam.height + th - 1) // th


def quat_to_rot(q) -> np.ndarray:
    q = _f64(q).reshape(4)
    R = np.zeros(9)
    _load().orc_quat_to_rot(_p(q, ctypes.c_double), _p(R, ctypes.c_double))
    return R.reshape(3, 3)


def sh_eval(deg: int, dirs):
    dirs = _f64(dirs).reshape(-1, 3)
    n = dirs.shape[0]
    D = (deg + 1) ** 2
    Y = np.zeros((n, D))
    dY = np.zeros((n, D, 3))
    _load().orc_sh_eval(deg, n, _p(dirs, ctypes.c_double), _p(Y, ctypes.c_double), _p(dY, ctypes.c_double))
    return Y, dY


def preprocess(g, cam, cfg: np.ndarray | None = None) -> dict:
    cfg = cfg_array() if cfg is None else cfg
    n, means, scales, quats, opac, sh, deg, st = _gauss_args(g)
    ca = cam_array(cam)
    out = dict(visible=np.zeros(n, np.int32), uv=np.zeros((n, 2)), depth=np.zeros(n),
               cov2d=np.zeros((n, 3)), conic=np.zeros((n, 3)), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), rgb=np.zeros((n, 3)), rgb_raw=np.zeros((n, 3)),
               amb=np.zeros(n, np.uint32), rect_in=np.zeros((n, 4), np.int32),
               rect_out=np.zeros((n, 4), np.int32))
    D, I32, U32 = ctypes.c_double, ctypes.c_int32, ctypes.c_uint32
    _load().orc_preprocess(n, _p(means, D), _p(scales, D), _p(quats, D), _p(opac, D), _p(sh, D), deg, st,
                           _p(ca, D), _p(cfg, D), _p(out["visible"], I32), _p(out["uv"], D),
                           _p(out["depth"], D), _p(out["cov2d"], D), _p(out["conic"], D),
                           _p(out["radius"], I32), _p(out["rect"], I32), _p(out["rgb"], D),
                           _p(out["rgb_raw"], D), _p(out["amb"], U32), _p(out["rect_in"], I32),
                           _p(out["rect_out"], I32))
    return out


def _mask_arg(cam, cfg, tile_mask):
    if tile_mask is None:
        return None
    TX, TY = tiles_xy(cam, cfg)
    m = np.ascontiguousarray(np.asarray(tile_mask, dtype=np.uint8).reshape(TX * TY))
    return m


def render_forward(g, cam, bg=(0.0, 0.0, 0.0), cfg: np.ndarray | None = None, tile_mask=None) -> dict:
    """Planar image [3, H, W], final transmittance [H, W], last contributor (1-based
    position in the tile list, 0 = none) [H, W] and its Gaussian index (-1 = none) [H, W];
    ``pix_dec`` [H, W]: bit (kind - 1) set for each kind of decision near its threshold at the
    pixel; ``alt``: one entry per such decision, with the pixel's colour, T and last Gaussian
    when that decision is taken the other way (``pix`` flat pixel index, ``kind``, ``g0``,
    ``g1`` the Gaussians involved); ``gauss_amb`` the per-Gaussian stage's bits."""
    cfg = cfg_array() if cfg is None else cfg
    n, means, scales, quats, opac, sh, deg, st = _gauss_args(g)
    ca = cam_array(cam)
    W, H = cam.width, cam.height
    bg = _f64(bg).reshape(3)
    m = _mask_arg(cam, cfg, tile_mask)
    D = ctypes.c_double
    cap = 4096
    while True:
        img = np.zeros((3, H, W))
        T = np.ones((H, W))
        last = np.zeros((H, W), np.int32)
        last_id = np.full((H, W), -1, np.int32)
        pix = np.zeros((H, W), np.uint8)
        gamb = np.zeros(n, np.uint32)
        a_pix = np.zeros(cap, np.int64)
        a_dec = np.zeros((cap, 3), np.int32)
        a_img = np.zeros((cap, 3))
        a_T = np.zeros(cap)
        a_last = np.zeros(cap, np.int32)
        counts = np.zeros(2, np.int64)
        _load().orc_render_forward(n, _p(means, D), _p(scales, D), _p(quats, D), _p(opac, D), _p(sh, D), deg, st,
                                   _p(ca, D), _p(cfg, D), _p(bg, D), _p(m, ctypes.c_uint8), _p(img, D), _p(T, D),
                                   _p(last, ctypes.c_int32), _p(last_id, ctypes.c_int32), _p(pix, ctypes.c_uint8),
                                   _p(gamb, ctypes.c_uint32), cap, _p(a_pix, ctypes.c_int64),
                                   _p(a_dec, ctypes.c_int32), _p(a_img, D), _p(a_T, D),
                                   _p(a_last, ctypes.c_int32), _p(counts, ctypes.c_long))
        k = int(counts[0])
        if k <= cap:
            break
        cap = k + 1024
    order = np.argsort(a_pix[:k], kind="stable")
    alt = dict(pix=a_pix[:k][order], kind=a_dec[:k, 0][order], g0=a_dec[:k, 1][order], g1=a_dec[:k, 2][order],
               img=a_img[:k][order], T=a_T[:k][order], last_id=a_last[:k][order])
    return dict(img=img, T=T, last=last, last_id=last_id, pix_dec=pix, gauss_amb=gamb, alt=alt,
                dec_overflow=int(counts[1]))


def render_backward(g, cam, dL_dimg, bg=(0.0, 0.0, 0.0), cfg: np.ndarray | None = None, tile_mask=None,
                    allowance: bool = True) -> dict:
    """Analytic FP64 gradients of L = <dL_dimg, image> w.r.t. every input, plus the
    screen-space gradients that the backward walk accumulates: mean2D (uv), conic, opacity,
    colour, and dL/dSigma' (cov2d: entries 00, 01, 11, full-matrix convention).  With
    ``allowance``, ``allow`` holds per Gaussian and per entry the summed magnitude of the changes
    that flipping each decision near its threshold makes to these gradients (keys as the
    gradients, plus ``opac2d`` for the screen-space opacity term); ``flips`` counts them; and
    ``cond`` the fp32 conditioning allowance of the chain rule (first-order effect of rounding
    R, J W, the camera-space mean and the view direction; zero for the screen-space terms)."""
    cfg = cfg_array() if cfg is None else cfg
    n, means, scales, quats, opac, sh, deg, st = _gauss_args(g)
    ca = cam_array(cam)
    W, H = cam.width, cam.height
    bg = _f64(bg).reshape(3)
    dimg = _f64(dL_dimg).reshape(3, H, W)
    m = _mask_arg(cam, cfg, tile_mask)
    out = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacities=np.zeros(n), sh=np.zeros_like(sh), uv=np.zeros((n, 2)), conic=np.zeros((n, 3)),
               rgb=np.zeros((n, 3)), cov2d=np.zeros((n, 3)), pix_dec=np.zeros((H, W), np.uint8),
               gauss_amb=np.zeros(n, np.uint32))
    al = cond = None
    if allowance:
        al = dict(screen=np.zeros((n, 9)), means=np.zeros((n, 3)), scales=np.zeros((n, 3)),
                  quats=np.zeros((n, 4)), opacities=np.zeros(n), sh=np.zeros_like(sh))
        cond = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)), sh=np.zeros_like(sh))
    counts = np.zeros(2, np.int64)
    D = ctypes.c_double
    A = (lambda k: _p(al[k], D)) if al is not None else (lambda k: None)
    Cd = (lambda k: _p(cond[k], D)) if cond is not None else (lambda k: None)
    _load().orc_render_backward(n, _p(means, D), _p(scales, D), _p(quats, D), _p(opac, D), _p(sh, D), deg, st,
                                _p(ca, D), _p(cfg, D), _p(bg, D), _p(m, ctypes.c_uint8), _p(dimg, D),
                                _p(out["means"], D), _p(out["scales"], D), _p(out["quats"], D),
                                _p(out["opacities"], D), _p(out["sh"], D), _p(out["uv"], D), _p(out["conic"], D),
                                _p(out["rgb"], D), _p(out["cov2d"], D), _p(out["pix_dec"], ctypes.c_uint8),
                                _p(out["gauss_amb"], ctypes.c_uint32), A("screen"), A("means"), A("scales"),
                                A("quats"), A("opacities"), A("sh"), Cd("means"), Cd("scales"), Cd("quats"),
                                Cd("sh"), _p(counts, ctypes.c_long))
    if al is not None:
        scr = al.pop("screen")
        al.update(uv=scr[:, 0:2], cov2d=scr[:, 2:5], opac2d=scr[:, 5], rgb=scr[:, 6:9])
        out["allow"] = al
        cond["opacities"] = np.zeros(n)
        for k in ("uv", "cov2d", "opac2d", "rgb"):
            cond[k] = np.zeros_like(al[k])
        out["cond"] = cond
    out["flips"] = int(counts[0])
    out["dec_overflow"] = int(counts[1])
    return out


class _Anisotropic:
    """An isotropic parameter set seen through the anisotropic definition."""

    def __init__(self, g):
        n = int(np.asarray(g.means).shape[0])
        s = _f64(g.scales).reshape(n)
        self.means, self.opacities, self.sh, self.sh_degree = g.means, g.opacities, g.sh, g.sh_degree
        self.scales = np.repeat(s[:, None], 3, axis=1)
        self.quats = np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (n, 1))


def render_forward_isotropic(g, cam, bg=(0.0, 0.0, 0.0), cfg: np.ndarray | None = None, tile_mask=None) -> dict:
    """The isotropic ablation of Sec. 7.3: one scale s per Gaussian for all three axes, so
    Sigma = s^2 I whatever the rotation; rendered as the anisotropic Gaussian with scales
    (s, s, s) and the identity rotation (g.scales is [n]; g.quats is not read)."""
    return render_forward(_Anisotropic(g), cam, bg, cfg, tile_mask)


def render_backward_isotropic(g, cam, dL_dimg, bg=(0.0, 0.0, 0.0), cfg: np.ndarray | None = None,
                              tile_mask=None) -> dict:
    """Gradients of the isotropic parameterisation: by the chain rule through s -> (s, s, s),
    dL/ds is the sum of the anisotropic dL/ds_k; the rotation has no effect (no quats entry)."""
    out = render_backward(_Anisotropic(g), cam, dL_dimg, bg, cfg, tile_mask)
    out["scales"] = out["scales"].sum(axis=1)
    del out["quats"]
    for key in ("allow", "cond"):
        if key in out:
            out[key]["scales"] = out[key]["scales"].sum(axis=1)
            del out[key]["quats"]
    return out


def reach_needed(g, cam, cfg: np.ndarray | None = None) -> np.ndarray:
    """Sorted keys i * tiles + t of the (Gaussian, tile) pairs any binning must keep: tiles of
    the Sec. 6 rectangle (under every rounding of it) in which some pixel centre certainly
    reaches alpha_min in FP64 (brute force over the tile's pixels)."""
    cfg = cfg_array() if cfg is None else cfg
    n, means, scales, quats, opac, sh, deg, st = _gauss_args(g)
    ca = cam_array(cam)
    D = ctypes.c_double
    cap = 1 << 20
    while True:
        out = np.zeros(cap, np.int64)
        k = _load().orc_reach_needed(n, _p(means, D), _p(scales, D), _p(quats, D), _p(opac, D), _p(sh, D), deg,
                                     st, _p(ca, D), _p(cfg, D), cap, _p(out, ctypes.c_int64))
        if k <= cap:
            return np.sort(out[:k])
        cap = k


def _bin_args(uv, depth, radius, chol, tau):
    uv = np.ascontiguousarray(np.asarray(uv, dtype=np.float32).reshape(-1, 2))
    n = uv.shape[0]
    depth = np.ascontiguousarray(np.asarray(depth if depth is not None else np.zeros(n), dtype=np.float32).reshape(-1))
    radius = np.ascontiguousarray(np.asarray(radius, dtype=np.int32).reshape(-1))
    if (chol is None) != (tau is None):
        raise ValueError("chol and tau go together")
    if chol is not None:
        chol = np.ascontiguousarray(np.asarray(chol, dtype=np.float32).reshape(n, 3))
        tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float32).reshape(n))
    return n, uv, depth, radius, chol, tau


def bin_instances(uv, depth, radius, width: int, height: int, tile_w: int = 16, tile_h: int = 16,
                  capacity: int | None = None, chol=None, tau=None):
    """Binning definition on given fp32 (u, v), fp32 depth and integer radius
    (radius <= 0: culled), over the 3-sigma tile rectangle, or, given the fp32 Cholesky factor
    (l11, l21, l22) of each conic and tau = 2 ln(o / alpha_min), over the tiles the
    reachable-tile rule keeps.  Returns (keys u64 [K], vals u32 [K], ranges u32 [T, 2])."""
    n, uv, depth, radius, chol, tau = _bin_args(uv, depth, radius, chol, tau)
    TX, TY = (width + tile_w - 1) // tile_w, (height + tile_h - 1) // tile_h
    ranges = np.zeros((TX * TY, 2), np.uint32)
    lib = _load()
    if capacity is None:
        capacity = instance_count(uv, radius, width, height, tile_w, tile_h, chol=chol, tau=tau)
    keys = np.zeros(max(capacity, 1), np.uint64)
    vals = np.zeros(max(capacity, 1), np.uint32)
    F = ctypes.c_float
    K = lib.orc_bin(n, _p(uv, F), _p(depth, F), _p(radius, ctypes.c_int32), _p(chol, F), _p(tau, F),
                    width, height, tile_w, tile_h, capacity, _p(keys, ctypes.c_uint64),
                    _p(vals, ctypes.c_uint32), _p(ranges, ctypes.c_uint32))
    if K < 0:
        raise OverflowError("instance count exceeds capacity")
    return keys[:K], vals[:K], ranges


def instance_count(uv, radius, width, height, tile_w=16, tile_h=16, chol=None, tau=None) -> int:
    """Number of (Gaussian, tile) instances, by the same rule as bin_instances."""
    n, uv, depth, radius, chol, tau = _bin_args(uv, None, radius, chol, tau)
    TX, TY = (width + tile_w - 1) // tile_w, (height + tile_h - 1) // tile_h
    ranges = np.zeros((TX * TY, 2), np.uint32)
    F = ctypes.c_float
    return int(_load().orc_bin(n, _p(uv, F), _p(depth, F), _p(radius, ctypes.c_int32), _p(chol, F), _p(tau, F),
                               width, height, tile_w, tile_h, 1 << 62, None, None, _p(ranges, ctypes.c_uint32)))

