"""Seeded synthetic Gaussian scenes, cameras and upstream gradients.

The workloads stand in for the paper's captured scenes (Mip-NeRF360, Tanks&Temples,
Deep Blending: 1-5 M Gaussians, 1080p, SH degree 3), which are not available here.
Every array is generated from numpy's PCG64 with a fixed seed (seed = 1000 * config +
k).  All floating-point values are float32 (what the rasterizer consumes); camera
parameters are rounded to float32 as well so that every consumer sees identical values.

Conventions: camera x right, y down, z forward; ``R`` and ``t`` map world to camera
(x_cam = R x_world + t); the world "up" direction is -y.  Quaternions are (r, i, j, k).
Opacities and scales are given already activated (sigmoid / exp applied here).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray          # (3, 3) world -> camera rotation, float32 values
    t: np.ndarray          # (3,)   world -> camera translation, float32 values
    near: float = 0.2

    def crop(self, x0: int, y0: int, width: int, height: int) -> "Camera":
        """The same pinhole restricted to the pixel window [x0, x0+width) x [y0, y0+height)."""
        return Camera(width, height, self.fx, self.fy, float(np.float32(self.cx - x0)),
                      float(np.float32(self.cy - y0)), self.R.copy(), self.t.copy(), self.near)


@dataclass
class Gaussians:
    means: np.ndarray      # (N, 3)
    scales: np.ndarray     # (N, 3), > 0
    quats: np.ndarray      # (N, 4), any non-zero norm
    opacities: np.ndarray  # (N,), in (0, 1)
    sh: np.ndarray         # (N, D, 3), D = (sh_degree + 1)^2 (or more: sh_stride)
    sh_degree: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Gaussians":
        return Gaussians(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                         self.opacities[idx].copy(), self.sh[idx].copy(), self.sh_degree, dict(self.meta))


def look_at_camera(eye, target, width: int, height: int, fov_x_deg: float, near: float = 0.2) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target``; horizontal field of view
    ``fov_x_deg``, square pixels, principal point at the image centre."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    down = np.array([0.0, 1.0, 0.0])
    right = np.cross(down, fwd)
    if np.linalg.norm(right) < 1e-9:  # looking straight up/down: pick any right vector
        right = np.cross(np.array([0.0, 0.0, 1.0]), fwd)
    right /= np.linalg.norm(right)
    dn = np.cross(fwd, right)
    R = np.stack([right, dn, fwd]).astype(np.float32).astype(np.float64)
    t = (-R @ eye).astype(np.float32).astype(np.float64)
    fx = float(np.float32(0.5 * width / math.tan(math.radians(fov_x_deg) / 2.0)))
    return Camera(width, height, fx, fx, float(np.float32(width / 2.0)), float(np.float32(height / 2.0)),
                  R, t, float(np.float32(near)))


def orbit_camera(radius: float, azimuth: float, elevation: float, width: int, height: int,
                 fov_x_deg: float = 60.0) -> Camera:
    """Camera on a sphere of ``radius`` around the origin, looking at the origin."""
    eye = radius * np.array([math.cos(elevation) * math.sin(azimuth), -math.sin(elevation),
                             -math.cos(elevation) * math.cos(azimuth)])
    return look_at_camera(eye, np.zeros(3), width, height, fov_x_deg)


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _sh_deg3(rng, n):
    """DC coefficients ~ U(0, 1), bands 1..3 ~ N(0, 0.05), as (N, 16, 3)."""
    sh = np.empty((n, 16, 3), dtype=np.float32)
    sh[:, 0, :] = rng.random((n, 3), dtype=np.float32)
    sh[:, 1:, :] = (0.05 * rng.standard_normal((n, 15, 3))).astype(np.float32)
    return sh


def _random_rotation(rng):
    """Haar-random rotation from the QR factorisation of a Gaussian matrix."""
    a = rng.standard_normal((3, 3))
    qm, rm = np.linalg.qr(a)
    qm = qm * np.sign(np.diag(rm))[None, :]
    if np.linalg.det(qm) < 0:
        qm[:, 0] = -qm[:, 0]
    return qm


def _cluster_means(rng, n, n_clusters=64, box=3.0):
    centres = rng.uniform(-box, box, (n_clusters, 3))
    rots = [_random_rotation(rng) for _ in range(n_clusters)]
    stds = rng.uniform(0.05, 0.5, (n_clusters, 3))
    which = rng.integers(0, n_clusters, n)
    z = rng.standard_normal((n, 3))
    out = np.empty((n, 3))
    for c in range(n_clusters):
        sel = which == c
        out[sel] = centres[c] + (z[sel] * stds[c]) @ rots[c].T
    return np.clip(out, -box, box)


def _uniform_ball(rng, n, r_in=0.0, r_out=1.0):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    u = rng.random(n)
    r = np.cbrt(r_in ** 3 + u * (r_out ** 3 - r_in ** 3))
    return d * r[:, None]


def _orbit_pose(rng):
    return float(rng.uniform(0.0, 2.0 * math.pi)), float(math.radians(rng.uniform(-30.0, 30.0)))


def _pack(means, log_scales, quats, opac_logits, sh, deg, **meta) -> Gaussians:
    return Gaussians(_f32(means), _f32(np.exp(log_scales)), _f32(quats), _f32(_sigmoid(opac_logits)),
                     _f32(sh), deg, meta)


def upstream_grad(seed: int, height: int, width: int) -> np.ndarray:
    """dL/dpixel ~ N(0, 1), planar (3, H, W) float32."""
    return _f32(_rng(seed).standard_normal((3, height, width)))


def config1(k: int = 1):
    """1,000 Gaussians, SH degree 0 (colour U(0,1) stored as the DC coefficient
    rgb / Y_00 with Y_00 = 1 / (2 sqrt(pi))), 128x128, fov 60 deg, camera at (0, 0, -4)
    looking at the origin, black background.  Forward only."""
    rng = _rng(1000 + k)
    n = 1000
    means = rng.uniform(-1.0, 1.0, (n, 3))
    log_s = rng.normal(-3.0, 0.5, (n, 3))
    quats = _unit_quats(rng, n)
    logit = rng.standard_normal(n)
    rgb = rng.random((n, 3))
    sh = (rgb * (2.0 * math.sqrt(math.pi)))[:, None, :]
    cam = look_at_camera([0.0, 0.0, -4.0], [0.0, 0.0, 0.0], 128, 128, 60.0)
    return _pack(means, log_s, quats, logit, sh, 0, name="config1"), cam, np.zeros(3, np.float32)


def config2(k: int = 1, n: int = 200_000):
    """200k Gaussians from 64 anisotropic clusters in [-3,3]^3, log-scales N(-4,1),
    SH degree 3, 1920x1080 camera on a radius-8 orbit; dL/dpixel ~ N(0,1)."""
    rng = _rng(2000 + k)
    means = _cluster_means(rng, n)
    log_s = rng.normal(-4.0, 1.0, (n, 3))
    quats = _unit_quats(rng, n)
    logit = rng.standard_normal(n)
    sh = _sh_deg3(rng, n)
    az, el = _orbit_pose(rng)
    cam = orbit_camera(8.0, az, el, 1920, 1080)
    g = _pack(means, log_s, quats, logit, sh, 3, name="config2")
    return g, cam, np.zeros(3, np.float32), upstream_grad(2100 + k, cam.height, cam.width)


def config2_crop(k: int = 1, n: int = 5000, crop: int = 64, margin: int = 16):
    """The gradient-check case: ``n`` Gaussians of the config-2 mixture whose means fall,
    seen through the 1080p camera, inside a centred ``crop`` x ``crop`` window widened by
    ``margin`` pixels; the camera is that window of the 1080p pinhole."""
    _, full, _, _ = config2(k, n=8)
    rng = _rng(2200 + k)
    lim = (crop / 2 + margin) / full.fx
    keep = []
    total = 0
    while total < n:
        m = _cluster_means(rng, 200_000)
        xc = m @ full.R.T + full.t
        ok = (xc[:, 2] > 0.5) & (np.abs(xc[:, 0] / xc[:, 2]) < lim) & (np.abs(xc[:, 1] / xc[:, 2]) < lim)
        keep.append(m[ok])
        total += int(ok.sum())
    means = np.concatenate(keep)[:n]
    log_s = rng.normal(-4.0, 1.0, (n, 3))
    quats = _unit_quats(rng, n)
    logit = rng.standard_normal(n)
    sh = _sh_deg3(rng, n)
    cam = full.crop(int(full.cx) - crop // 2, int(full.cy) - crop // 2, crop, crop)
    g = _pack(means, log_s, quats, logit, sh, 3, name="config2_crop")
    return g, cam, np.zeros(3, np.float32), upstream_grad(2300 + k, crop, crop)


def _unbounded(rng, n, frac_inner=0.8):
    n_in = int(round(frac_inner * n))
    n_out = n - n_in
    means = np.concatenate([_uniform_ball(rng, n_in, 0.0, 1.0), _uniform_ball(rng, n_out, 5.0, 50.0)])
    log_s = np.concatenate([rng.normal(-5.0, 1.0, (n_in, 3)), rng.normal(-2.0, 1.0, (n_out, 3))])
    quats = _unit_quats(rng, n)
    logit = rng.normal(0.0, 1.5, n)
    sh = _sh_deg3(rng, n)
    return means, log_s, quats, logit, sh


def config3(k: int = 1, n: int = 3_000_000, width: int = 1920, height: int = 1080):
    """Large unbounded scene: 80% of means uniform in the unit ball (log-scale N(-5,1)),
    20% in the shell 5 <= r <= 50 (uniform in volume, log-scale N(-2,1)); opacity
    sigmoid(N(0,1.5)); SH degree 3; 1920x1080 camera on a radius-3 orbit; dL/dpixel ~ N(0,1)."""
    rng = _rng(3000 + k)
    means, log_s, quats, logit, sh = _unbounded(rng, n)
    az, el = _orbit_pose(rng)
    cam = orbit_camera(3.0, az, el, width, height)
    g = _pack(means, log_s, quats, logit, sh, 3, name="config3")
    return g, cam, np.zeros(3, np.float32), upstream_grad(3100 + k, cam.height, cam.width)


RESOLUTIONS = [(640, 480), (1280, 720), (1600, 900), (1920, 1080)]


def config4(k: int = 1, n: int = 1_000_000, views: int = 16):
    """One scene with the config-3 distribution (1M Gaussians) and ``views`` cameras of
    uneven resolution on radius-3 orbit poses (azimuth U[0, 2pi), elevation U[-30, 30] deg)."""
    rng = _rng(4000 + k)
    means, log_s, quats, logit, sh = _unbounded(rng, n)
    g = _pack(means, log_s, quats, logit, sh, 3, name="config4")
    cams, grads = [], []
    for v in range(views):
        w, h = RESOLUTIONS[int(rng.integers(0, len(RESOLUTIONS)))]
        az, el = _orbit_pose(rng)
        cams.append(orbit_camera(3.0, az, el, w, h))
        grads.append(upstream_grad(4100 + 100 * k + v, h, w))
    return g, cams, np.zeros(3, np.float32), grads


def config5(k: int = 1, scenes: int = 8, views: int = 4, n_min: int = 50_000, n_max: int = 2_000_000):
    """``scenes`` independent cluster-mixture scenes with log-uniform Gaussian counts in
    [n_min, n_max], SH degree 3, ``views`` cameras each at mixed resolutions."""
    rng = _rng(5000 + k)
    out = []
    for s in range(scenes):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        means = _cluster_means(rng, n)
        log_s = rng.normal(-4.0, 1.0, (n, 3))
        quats = _unit_quats(rng, n)
        logit = rng.standard_normal(n)
        sh = _sh_deg3(rng, n)
        g = _pack(means, log_s, quats, logit, sh, 3, name=f"config5_scene{s}")
        cams, grads = [], []
        for v in range(views):
            w, h = RESOLUTIONS[int(rng.integers(0, len(RESOLUTIONS)))]
            az, el = _orbit_pose(rng)
            cams.append(orbit_camera(8.0, az, el, w, h))
            grads.append(upstream_grad(5100 + 1000 * k + 10 * s + v, h, w))
        out.append((g, cams, grads))
    return out, np.zeros(3, np.float32)


def tiny_scene(seed: int, n: int = 64, width: int = 48, height: int = 40, deg: int = 3,
               log_scale_mean: float = -2.5, log_scale_std: float = 0.5, box: float = 0.8,
               distance: float = 3.0, fov_x_deg: float = 60.0, unnormalised_quats: bool = True,
               opacity_logit_std: float = 1.0):
    """Small scene in front of a camera at (0, 0, -distance): for unit and parity tests
    that must span several tiles and a ragged image edge."""
    rng = _rng(seed)
    means = rng.uniform(-box, box, (n, 3))
    log_s = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    quats = _unit_quats(rng, n)
    if unnormalised_quats:
        quats = quats * rng.uniform(0.5, 2.0, (n, 1))
    logit = rng.normal(0.0, opacity_logit_std, n)
    D = (deg + 1) ** 2
    sh = np.empty((n, D, 3))
    sh[:, 0, :] = rng.random((n, 3))
    if D > 1:
        sh[:, 1:, :] = 0.1 * rng.standard_normal((n, D - 1, 3))
    cam = look_at_camera([0.0, 0.0, -distance], [0.0, 0.0, 0.0], width, height, fov_x_deg)
    return _pack(means, log_s, quats, logit, sh, deg, name=f"tiny{seed}"), cam


def density_state(seed: int, n: int, deg: int = 3):
    """Optimiser state at a refinement (Sec. 5.2): raw parameters (log scales, logit
    opacities), Adam moments, view-space gradient statistics and the two standard normal
    draws per Gaussian that a split consumes.  The spreads put every decision (prune, keep,
    clone, split) in play at the default thresholds with tau_S around 0.01 to 0.05."""
    rng = _rng(seed)
    D = (deg + 1) ** 2
    params = dict(means=rng.uniform(-3, 3, (n, 3)), log_scales=rng.normal(-4.0, 1.2, (n, 3)),
                  quats=_unit_quats(rng, n) * rng.uniform(0.5, 2.0, (n, 1)),
                  logit_opacities=rng.normal(-1.0, 2.5, n), sh=0.3 * rng.standard_normal((n, D, 3)))
    m = {k: 1e-3 * rng.standard_normal(a.shape) for k, a in params.items()}
    v = {k: 1e-6 * rng.random(a.shape) for k, a in params.items()}
    count = rng.integers(0, 40, n).astype(np.float64)
    accum = count * rng.lognormal(np.log(2e-4), 0.8, n)
    max_radius = np.floor(rng.exponential(8.0, n)) * (count > 0)
    normals = rng.standard_normal((n, 2, 3))
    f = {k: _f32(a) for k, a in params.items()}
    return (f, {k: _f32(a) for k, a in m.items()}, {k: _f32(a) for k, a in v.items()}, _f32(accum), _f32(count),
            _f32(max_radius), _f32(normals))
