"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics, not by
the oracle itself: closed forms, textbook/library routines, published constants, exact
binary-fraction worked examples, brute force and finite differences.

Each test names the passage of the paper whose formula it pins.
"""
import math
import os

import numpy as np
import pytest

import oracle
from synthetic import Gaussians, look_at_camera, tiny_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Y00 = 0.5 / math.sqrt(math.pi)


def _gauss(means, scales, quats, opac, rgb=None, sh=None, deg=0):
    means = np.asarray(means, np.float64).reshape(-1, 3)
    n = means.shape[0]
    if sh is None:
        rgb = np.asarray(rgb, np.float64).reshape(n, 3)
        sh = (rgb / Y00)[:, None, :]
    return Gaussians(means, np.asarray(scales, np.float64).reshape(n, 3), np.asarray(quats, np.float64).reshape(n, 4),
                     np.asarray(opac, np.float64).reshape(n), np.asarray(sh, np.float64), deg)


def _axis_cam(width, height, distance=4.0, fov=60.0):
    """Camera at (0, 0, -distance) looking down +z: R = I, t = (0, 0, distance)."""
    return look_at_camera([0.0, 0.0, -distance], [0.0, 0.0, 0.0], width, height, fov)


# --------------------------------------------------------------------------------------
# eq. quat (App. A): rotation of a unit quaternion
# --------------------------------------------------------------------------------------
def _rodrigues(axis, angle):
    n = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -n[2], n[1]], [n[2], 0, -n[0]], [-n[1], n[0], 0]])
    return np.eye(3) * math.cos(angle) + math.sin(angle) * K + (1 - math.cos(angle)) * np.outer(n, n)


@pytest.mark.parametrize("seed", range(6))
def test_quat_rotation_matches_rodrigues(seed):
    rng = np.random.default_rng(seed)
    axis = rng.standard_normal(3)
    angle = rng.uniform(-math.pi, math.pi)
    n = axis / np.linalg.norm(axis)
    q = np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * n])
    R = oracle.quat_to_rot(q)
    np.testing.assert_allclose(R, _rodrigues(axis, angle), atol=1e-14)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1.0) < 1e-13
    np.testing.assert_allclose(oracle.quat_to_rot(-q), R, atol=1e-14)


# --------------------------------------------------------------------------------------
# Sec. 4, eq. volume-render: Sigma = R S S^T R^T and its EWA projection
# --------------------------------------------------------------------------------------
def test_ewa_isotropic_on_axis_closed_form():
    """Isotropic Gaussian (std s) on the optical axis at depth z:
    Sigma' = ((f s / z)^2 + 0.3) I, conic = I / that, radius = ceil(3 sqrt(that))."""
    cam = _axis_cam(128, 96)
    s, z = 0.05, 4.0
    g = _gauss([[0, 0, 0]], [[s, s, s]], [[0.3, -0.2, 0.9, 0.1]], [0.7], rgb=[[0.2, 0.4, 0.6]])
    pp = oracle.preprocess(g, cam)
    var = (cam.fx * s / z) ** 2 + 0.3
    np.testing.assert_allclose(pp["cov2d"][0], [var, 0.0, var], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pp["conic"][0], [1 / var, 0.0, 1 / var], rtol=1e-13, atol=1e-13)
    assert pp["radius"][0] == math.ceil(3 * math.sqrt(var))
    np.testing.assert_allclose(pp["uv"][0], [cam.cx, cam.cy], atol=1e-12)
    assert pp["depth"][0] == pytest.approx(z, abs=1e-12)


@pytest.mark.parametrize("xy", [(0.3, -0.2), (-0.5, 0.4), (0.7, 0.1)])
def test_ewa_isotropic_off_axis_hand_jacobian(xy):
    """Off axis: Sigma' = s^2 J J^T + 0.3 I with the perspective Jacobian
    J = [[f/z, 0, -f x/z^2], [0, f/z, -f y/z^2]] written out by hand."""
    cam = _axis_cam(256, 256)
    x, y = xy
    s, zc = 0.04, 4.0 + 0.5
    g = _gauss([[x, y, 0.5]], [[s, s, s]], [[1, 0, 0, 0]], [0.5], rgb=[[0.5, 0.5, 0.5]])
    pp = oracle.preprocess(g, cam)
    f = cam.fx
    JJt00 = f * f / zc ** 2 + f * f * x * x / zc ** 4
    JJt01 = f * f * x * y / zc ** 4
    JJt11 = f * f / zc ** 2 + f * f * y * y / zc ** 4
    np.testing.assert_allclose(pp["cov2d"][0], [s * s * JJt00 + 0.3, s * s * JJt01, s * s * JJt11 + 0.3], rtol=1e-12)
    np.testing.assert_allclose(pp["uv"][0], [f * x / zc + cam.cx, f * y / zc + cam.cy], rtol=1e-14)


def test_ewa_anisotropic_axes_follow_quaternion():
    """Axis-aligned ellipsoid diag(a, b, c) at the optical axis: the identity quaternion
    projects (a, b); a 90 deg turn about z swaps them; a 90 deg turn about x shows (a, c)."""
    cam = _axis_cam(128, 128)
    a, b, c, z = 0.03, 0.07, 0.11, 4.0
    h = math.sqrt(0.5)
    qs = [[1, 0, 0, 0], [h, 0, 0, h], [h, h, 0, 0]]
    g = _gauss([[0, 0, 0]] * 3, [[a, b, c]] * 3, qs, [0.5] * 3, rgb=[[0.5] * 3] * 3)
    pp = oracle.preprocess(g, cam)
    k = (cam.fx / z) ** 2
    expect = [[k * a * a + 0.3, k * b * b + 0.3], [k * b * b + 0.3, k * a * a + 0.3], [k * a * a + 0.3, k * c * c + 0.3]]
    for i in range(3):
        np.testing.assert_allclose(pp["cov2d"][i][[0, 2]], expect[i], rtol=1e-12)
        assert abs(pp["cov2d"][i][1]) < 1e-12


def test_covariance_invariant_under_quaternion_scale_and_sign():
    g, cam = tiny_scene(11, n=32, unnormalised_quats=False)
    ref = oracle.preprocess(g, cam)
    for factor in (-1.0, 0.25, 7.5):
        g2 = Gaussians(g.means, g.scales, g.quats.astype(np.float64) * factor, g.opacities, g.sh, g.sh_degree)
        pp = oracle.preprocess(g2, cam)
        np.testing.assert_allclose(pp["cov2d"], ref["cov2d"], rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(pp["radius"], ref["radius"])


def test_covariance_is_symmetric_positive_definite():
    g, cam = tiny_scene(12, n=200)
    pp = oracle.preprocess(g, cam)
    A, B, C = pp["cov2d"][:, 0], pp["cov2d"][:, 1], pp["cov2d"][:, 2]
    vis = pp["visible"] > 0
    assert vis.sum() > 100
    assert np.all(A[vis] > 0.3 - 1e-12) and np.all(C[vis] > 0.3 - 1e-12)
    det = A * C - B * B
    assert np.all(det[vis] >= 0.09 - 1e-9)   # dilation bounds the determinant from below


# --------------------------------------------------------------------------------------
# SH colour (Sec. 4, Sec. 7.1): real SH basis, 4 bands
# --------------------------------------------------------------------------------------
def _scipy_real_sh(deg, dirs):
    from scipy import special
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    out = np.zeros((dirs.shape[0], (deg + 1) ** 2))
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            if hasattr(special, "sph_harm_y"):
                Yc = special.sph_harm_y(l, abs(m), theta, phi)
            else:  # older scipy: sph_harm(m, n, azimuth, polar)
                Yc = special.sph_harm(abs(m), l, phi, theta)
            k = l * l + l + m
            if m > 0:
                out[:, k] = math.sqrt(2) * Yc.real
            elif m < 0:
                out[:, k] = math.sqrt(2) * Yc.imag
            else:
                out[:, k] = Yc.real
    return out


def _rand_dirs(seed, n):
    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_basis_matches_scipy():
    dirs = _rand_dirs(0, 500)
    Y, _ = oracle.sh_eval(3, dirs)
    np.testing.assert_allclose(Y, _scipy_real_sh(3, dirs), atol=1e-12)


def test_sh_basis_matches_published_constants():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "sh_constants_sloan2008.txt")) if ln.strip() and ln[0] != "#"]
    dirs = _rand_dirs(1, 64)
    Y, _ = oracle.sh_eval(3, dirs)
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    polys = {"1": np.ones_like(x), "y": y, "z": z, "x": x, "xy": x * y, "yz": y * z, "3zz-1": 3 * z * z - 1,
             "xz": x * z, "xx-yy": x * x - y * y, "y(3xx-yy)": y * (3 * x * x - y * y), "xyz": x * y * z,
             "y(5zz-1)": y * (5 * z * z - 1), "z(5zz-3)": z * (5 * z * z - 3), "x(5zz-1)": x * (5 * z * z - 1),
             "z(xx-yy)": z * (x * x - y * y), "x(xx-3yy)": x * (x * x - 3 * y * y)}
    for k, l, m, c, p in rows:
        np.testing.assert_allclose(Y[:, int(k)], float(c) * polys[p], atol=6e-7 * 10, rtol=2e-6)


def test_sh_basis_orthonormal_by_quadrature():
    zs, wz = np.polynomial.legendre.leggauss(8)
    nphi = 16
    phis = 2 * math.pi * np.arange(nphi) / nphi
    Z, P = np.meshgrid(zs, phis, indexing="ij")
    Wq = np.repeat(wz[:, None], nphi, axis=1) * (2 * math.pi / nphi)
    s = np.sqrt(1 - Z ** 2)
    dirs = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    Y, _ = oracle.sh_eval(3, dirs)
    G = (Y * Wq.reshape(-1, 1)).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_gradient_matches_tangent_finite_difference():
    dirs = _rand_dirs(2, 40)
    _, dY = oracle.sh_eval(3, dirs)
    rng = np.random.default_rng(3)
    h = 1e-6
    for i in range(dirs.shape[0]):
        d = dirs[i]
        e = rng.standard_normal(3)
        e -= d * (d @ e)
        dp = (d + h * e) / np.linalg.norm(d + h * e)
        dm = (d - h * e) / np.linalg.norm(d - h * e)
        fd = (oracle.sh_eval(3, dp[None])[0][0] - oracle.sh_eval(3, dm[None])[0][0]) / (2 * h)
        np.testing.assert_allclose(dY[i] @ e, fd, atol=1e-7)


def test_sh_degree0_is_constant_colour():
    g, cam = tiny_scene(13, n=50, deg=0)
    pp = oracle.preprocess(g, cam)
    np.testing.assert_allclose(pp["rgb"], np.maximum(g.sh[:, 0, :].astype(np.float64) * Y00, 0), rtol=1e-12)


# --------------------------------------------------------------------------------------
# eq. front-to-back + App. C rules
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("sig,opac,rgb,bg", [(3.1, 0.8, (0.9, 0.3, 0.1), (0, 0, 0)),
                                             (1.2, 0.5, (0.2, 0.8, 0.4), (1, 1, 1)),
                                             (6.3, 0.995, (0.7, 0.6, 0.5), (0.25, 0.5, 0.75))])
def test_single_gaussian_analytic_footprint(sig, opac, rgb, bg):
    """One isotropic Gaussian: every pixel is bg (1 - a) + a c with
    a = min(0.99, o exp(-rho^2 / (2 sigma'^2))), and bg where a < 1/255."""
    cam = _axis_cam(128, 128)
    z = 4.0
    s = math.sqrt(sig * sig - 0.3) * z / cam.fx
    g = _gauss([[0, 0, 0]], [[s, s, s]], [[1, 0, 0, 0]], [opac], rgb=[rgb])
    out = oracle.render_forward(g, cam, bg)
    py, px = np.mgrid[0:128, 0:128]
    rho2 = (px + 0.5 - cam.cx) ** 2 + (py + 0.5 - cam.cy) ** 2
    a = np.minimum(0.99, opac * np.exp(-rho2 / (2 * sig * sig)))
    a = np.where(a < 1 / 255, 0.0, a)
    for ch in range(3):
        np.testing.assert_allclose(out["img"][ch], bg[ch] * (1 - a) + a * rgb[ch], atol=1e-12)
    np.testing.assert_allclose(out["T"], 1 - a, atol=1e-12)
    np.testing.assert_array_equal(out["last"], (a > 0).astype(np.int32))


def test_stop_rule_stack_of_half_alpha_splats():
    """App. C: stop before the accumulated opacity exceeds 0.9999 (golden worked example)."""
    gold = dict(ln.split() for ln in open(os.path.join(GOLDEN, "stop_rule_stack.txt")) if ln.strip() and ln[0] != "#")
    n = int(gold["n_splats"])
    cam = _axis_cam(33, 33)    # principal point 16.5: pixel (16, 16) sits on the optical axis
    depths = 2.0 + 0.1 * np.arange(n)
    means = np.stack([np.zeros(n), np.zeros(n), depths - 4.0], 1)
    s = 0.02
    c, bg = 0.75, 0.5
    g = _gauss(means, [[s, s, s]] * n, [[1, 0, 0, 0]] * n, [float(gold["alpha"])] * n, rgb=[[c, c, c]] * n)
    out = oracle.render_forward(g, cam, (bg, bg, bg))
    assert out["last"][16, 16] == int(gold["blended"])
    assert out["T"][16, 16] == float(gold["T_final"])
    f = float(gold["colour_factor"])
    np.testing.assert_allclose(out["img"][:, 16, 16], c * f + bg * (1 - f), atol=1e-15)


def test_no_gaussians_gives_background():
    cam = _axis_cam(40, 24)
    g = _gauss(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 4)), np.zeros(0), rgb=np.zeros((0, 3)))
    out = oracle.render_forward(g, cam, (0.1, 0.2, 0.3))
    for ch, b in enumerate((0.1, 0.2, 0.3)):
        assert np.all(out["img"][ch] == b)
    assert np.all(out["T"] == 1.0) and np.all(out["last"] == 0)


def test_alpha_below_threshold_has_no_effect():
    cam = _axis_cam(64, 64)
    g = _gauss([[0, 0, 0]], [[0.2, 0.2, 0.2]], [[1, 0, 0, 0]], [0.999 / 255], rgb=[[1, 1, 1]])
    out = oracle.render_forward(g, cam, (0.3, 0.3, 0.3))
    assert np.all(out["img"] == 0.3) and np.all(out["T"] == 1.0)


def test_opacity_clamp_gives_99_percent():
    cam = _axis_cam(33, 33)
    g = _gauss([[0, 0, 0]], [[0.3, 0.3, 0.3]], [[1, 0, 0, 0]], [0.9999], rgb=[[0.8, 0.8, 0.8]])
    out = oracle.render_forward(g, cam, (0.1, 0.1, 0.1))
    np.testing.assert_allclose(out["img"][:, 16, 16], 0.99 * 0.8 + 0.01 * 0.1, atol=1e-14)


def test_white_splats_telescoping_identity():
    """With every colour 1 and a black background, sum_i T_i a_i = 1 - T_final
    (eq. front-to-back with T_{i+1} = T_i (1 - a_i))."""
    g, cam = tiny_scene(21, n=120, deg=0, width=64, height=48)
    g.sh[:] = 1.0 / Y00
    out = oracle.render_forward(g, cam)
    for ch in range(3):
        np.testing.assert_allclose(out["img"][ch], 1 - out["T"], atol=1e-12)
    assert np.all(out["T"] >= 1e-4)


def test_background_enters_through_final_transmittance():
    g, cam = tiny_scene(22, n=80, width=48, height=40)
    a = oracle.render_forward(g, cam, (0, 0, 0))
    b = oracle.render_forward(g, cam, (0.2, 0.5, 0.9))
    for ch, bgc in enumerate((0.2, 0.5, 0.9)):
        np.testing.assert_allclose(b["img"][ch], a["img"][ch] + bgc * a["T"], atol=1e-12)


def test_non_overlapping_splats_are_order_independent():
    """Splats whose footprints (alpha >= 1/255) do not overlap give the same image for any
    depth order: each pixel then blends at most one splat."""
    cam = _axis_cam(64, 64)
    grid = [(u, v) for u in (12.0, 28.0, 44.0) for v in (10.0, 30.0, 50.0)]
    n = len(grid)
    rng = np.random.default_rng(5)
    rgb = rng.random((n, 3))
    sig_px = 1.5

    def scene(depths):
        means, scales = [], []
        for (u, v), z in zip(grid, depths):
            means.append([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z - 4.0])
            s = sig_px * z / cam.fx           # same projected footprint at every depth
            scales.append([s, s, s])
        return _gauss(means, scales, [[1, 0, 0, 0]] * n, [0.8] * n, rgb=rgb)

    ref = oracle.render_forward(scene(np.linspace(3.0, 5.0, n)), cam)
    for seed in range(3):
        depths = np.random.default_rng(seed).permutation(np.linspace(3.0, 5.0, n))
        out = oracle.render_forward(scene(depths), cam)
        np.testing.assert_allclose(out["img"], ref["img"], atol=1e-12)
        np.testing.assert_allclose(out["T"], ref["T"], atol=1e-12)
    assert np.count_nonzero(ref["last"]) > 9 * 20


def test_front_to_back_order_by_depth_not_index():
    """Eq. front-to-back: the nearer splat is blended first, whatever its index.
    Two splats centred on the pixel with alpha = 0.5: C = 0.5 c_near + 0.25 c_far."""
    cam = _axis_cam(33, 33)
    s = 0.05
    red, blue = [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]
    for near_first in (True, False):
        zs = [-1.0, 1.0] if near_first else [1.0, -1.0]
        cols = [red, blue] if near_first else [blue, red]
        g = _gauss([[0, 0, zs[0]], [0, 0, zs[1]]], [[s, s, s], [s, s, s]], [[1, 0, 0, 0]] * 2, [0.5, 0.5], rgb=cols)
        out = oracle.render_forward(g, cam)
        np.testing.assert_allclose(out["img"][:, 16, 16], [0.5, 0.0, 0.25], atol=1e-15)
        assert out["T"][16, 16] == 0.25


@pytest.mark.parametrize("inside", [True, False])
def test_guard_band_and_near_plane_reject(inside):
    """Sec. 6 guard band (reading: reject when |x/z| > 1.3 tan(fov_x/2), same in y) and
    near plane (reject when z <= 0.2)."""
    cam = _axis_cam(64, 48)
    z = 4.0
    f = 1.0 - 1e-3 if inside else 1.0 + 1e-3
    tx, ty = 1.3 * 32 / cam.fx, 1.3 * 24 / cam.fy
    means = [[f * tx * z, 0, 0], [0, f * ty * z, 0], [-f * tx * z, 0, 0],
             [0, 0, (0.2 * (1 + 1e-3) if inside else 0.2 * (1 - 1e-3)) - 4.0]]
    s = 2.0   # large enough to reach the screen from outside the guard band
    g = _gauss(means, [[s, s, s]] * 4, [[1, 0, 0, 0]] * 4, [0.5] * 4, rgb=[[1, 1, 1]] * 4)
    pp = oracle.preprocess(g, cam)
    assert list(pp["visible"]) == ([1, 1, 1, 1] if inside else [0, 0, 0, 0])


def test_transmittance_monotone_when_adding_a_splat_behind():
    g, cam = tiny_scene(23, n=60, width=48, height=40)
    ref = oracle.render_forward(g, cam)
    g2 = Gaussians(np.concatenate([g.means, [[0.0, 0.0, 0.95]]]).astype(np.float32),
                   np.concatenate([g.scales, [[0.4, 0.4, 0.4]]]).astype(np.float32),
                   np.concatenate([g.quats, [[1, 0, 0, 0]]]).astype(np.float32),
                   np.concatenate([g.opacities, [0.9]]).astype(np.float32),
                   np.concatenate([g.sh, np.full((1,) + g.sh.shape[1:], 0.1)]).astype(np.float32), g.sh_degree)
    out = oracle.render_forward(g2, cam)
    assert np.all(out["T"] <= ref["T"] + 1e-15)
    assert np.any(out["T"] < ref["T"] - 1e-3)


# --------------------------------------------------------------------------------------
# App. C / Algorithm 2 binning: keys, one stable sort, tile ranges
# --------------------------------------------------------------------------------------
def _random_screen(seed, n, W, H):
    rng = np.random.default_rng(seed)
    uv = np.stack([rng.uniform(-40, W + 40, n), rng.uniform(-40, H + 40, n)], 1).astype(np.float32)
    depth = rng.uniform(0.2, 30, n).astype(np.float32)
    depth[rng.random(n) < 0.1] = depth[0]          # exact depth ties
    radius = rng.integers(1, 60, n).astype(np.int32)
    radius[rng.random(n) < 0.1] = 0                # culled
    return uv, depth, radius


@pytest.mark.parametrize("seed,W,H,tw,th", [(0, 100, 70, 16, 16), (1, 64, 64, 16, 16), (2, 90, 50, 8, 8), (3, 77, 33, 16, 8)])
def test_binning_matches_brute_force(seed, W, H, tw, th):
    n = 300
    uv, depth, radius = _random_screen(seed, n, W, H)
    keys, vals, ranges = oracle.bin_instances(uv, depth, radius, W, H, tw, th)
    TX, TY = -(-W // tw), -(-H // th)
    dbits = depth.view(np.uint32)
    # brute force per tile: the square [u - r, u + r] x [v - r, v + r] overlaps the tile's
    # pixel span [tw*tx, tw*(tx+1)) x [th*ty, th*(ty+1)); order by (fp32 depth bits, index)
    for t in range(TX * TY):
        tx, ty = t % TX, t // TX
        sel = [i for i in range(n) if radius[i] > 0
               and uv[i, 0] - radius[i] < tw * (tx + 1) and uv[i, 0] + radius[i] >= tw * tx
               and uv[i, 1] - radius[i] < th * (ty + 1) and uv[i, 1] + radius[i] >= th * ty]
        sel.sort(key=lambda i: (int(dbits[i]), i))
        a, b = ranges[t]
        assert list(vals[a:b]) == sel, t
        assert np.all(keys[a:b] >> np.uint64(32) == t)
        assert np.all((keys[a:b] & np.uint64(0xFFFFFFFF)) == dbits[vals[a:b]])
    # the whole array is the stable sort of the emitted keys
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])


def test_binning_empty_and_capacity():
    uv = np.zeros((0, 2), np.float32)
    keys, vals, ranges = oracle.bin_instances(uv, np.zeros(0, np.float32), np.zeros(0, np.int32), 50, 50)
    assert keys.size == 0 and np.all(ranges == 0)
    uv, depth, radius = _random_screen(9, 50, 64, 64)
    with pytest.raises(OverflowError):
        oracle.bin_instances(uv, depth, radius, 64, 64, capacity=3)


# --------------------------------------------------------------------------------------
# Sec. 6 backward + App. A: analytic gradients vs central finite differences
# --------------------------------------------------------------------------------------
def _loss(g, cam, dimg, bg):
    return float(np.sum(oracle.render_forward(g, cam, bg)["img"] * dimg))


def _fd_check(g, cam, dimg, bg, params, rel_tol=1e-5):
    ana = oracle.render_backward(g, cam, dimg, bg)
    names = {"means": "means", "scales": "scales", "quats": "quats", "opacities": "opacities", "sh": "sh"}
    checked = skipped = 0
    worst = 0.0
    for name, idx in params:
        arr = getattr(g, names[name])
        theta = float(arr[idx])
        h = 1e-6 * max(1.0, abs(theta))
        vals = []
        for hh in (h, h / 4):
            arr[idx] = theta + hh
            lp = _loss(g, cam, dimg, bg)
            arr[idx] = theta - hh
            lm = _loss(g, cam, dimg, bg)
            arr[idx] = theta
            vals.append((lp - lm) / (2 * hh))
        fd, fd2 = vals
        scale = max(1e-3 * np.max(np.abs(ana[name])), abs(fd))
        if abs(fd - fd2) > 1e-6 * max(scale, 1e-8) + 1e-9:
            skipped += 1        # a discrete decision flips inside [theta - h, theta + h]
            continue
        err = abs(ana[name][idx] - fd) / max(scale, 1e-12)
        worst = max(worst, err)
        assert err <= rel_tol, (name, idx, ana[name][idx], fd)
        checked += 1
    return checked, skipped, worst


def test_backward_matches_finite_differences_tiny():
    g, cam = tiny_scene(31, n=10, width=24, height=24, deg=3, log_scale_mean=-2.2)
    g = Gaussians(*(np.array(a, np.float64) for a in (g.means, g.scales, g.quats, g.opacities, g.sh)), g.sh_degree)
    dimg = np.random.default_rng(32).standard_normal((3, 24, 24))
    bg = (0.1, 0.3, 0.2)
    params = []
    for i in range(g.n):
        params += [("means", (i, k)) for k in range(3)] + [("scales", (i, k)) for k in range(3)]
        params += [("quats", (i, k)) for k in range(4)] + [("opacities", (i,))]
        params += [("sh", (i, k, c)) for k in range(16) for c in range(3)]
    checked, skipped, worst = _fd_check(g, cam, dimg, bg, params)
    assert checked >= 0.9 * len(params), (checked, skipped)


def test_backward_matches_finite_differences_config2_crop():
    """The config-2 gradient-check case (5k Gaussians of the cluster mixture seen through a
    64x64 window of the 1080p camera): FD on every parameter of a few Gaussians that
    touch the image, plus random scalars."""
    from synthetic import config2_crop
    g, cam, bg, dimg = config2_crop()
    g = Gaussians(*(np.array(a, np.float64) for a in (g.means, g.scales, g.quats, g.opacities, g.sh)), g.sh_degree)
    ana = oracle.render_backward(g, cam, dimg, bg)
    touched = np.nonzero(np.abs(ana["opacities"]) > 0)[0]
    assert touched.size > 50
    rng = np.random.default_rng(7)
    pick = rng.choice(touched, 6, replace=False)
    params = []
    for i in pick:
        params += [("means", (i, k)) for k in range(3)] + [("scales", (i, k)) for k in range(3)]
        params += [("quats", (i, k)) for k in range(4)] + [("opacities", (i,))]
        params += [("sh", (i, k, c)) for k in (0, 1, 5, 12) for c in range(3)]
    for _ in range(60):
        i = int(rng.choice(touched))
        name = ["means", "scales", "quats", "opacities", "sh"][int(rng.integers(0, 5))]
        if name == "opacities":
            params.append((name, (i,)))
        elif name == "sh":
            params.append((name, (i, int(rng.integers(0, 16)), int(rng.integers(0, 3)))))
        else:
            params.append((name, (i, int(rng.integers(0, 4 if name == "quats" else 3)))))
    checked, skipped, worst = _fd_check(g, cam, dimg, bg, params)
    assert checked >= 0.85 * len(params), (checked, skipped)


# --------------------------------------------------------------------------------------
# Reachable-tile rule (a refinement of the Sec. 6 rectangle): pinned against FP64 brute
# force over pixel centres, not against its own fp32 steps.
# --------------------------------------------------------------------------------------
from screen_util import ALPHA_MIN, random_splats  # noqa: E402


def _rect_tiles(uv, r, W, H, tw, th):
    TX, TY = -(-W // tw), -(-H // th)
    fu, fv = int(np.floor(uv[0])), int(np.floor(uv[1]))
    x0 = min(max((fu - r) // tw, 0), TX); x1 = min(max((fu + r) // tw + 1, 0), TX)
    y0 = min(max((fv - r) // th, 0), TY); y1 = min(max((fv + r) // th + 1, 0), TY)
    return x0, x1, y0, y1


@pytest.mark.parametrize("seed,W,H,tw,th,rmax", [(11, 160, 96, 16, 16, 60), (12, 120, 72, 8, 8, 30),
                                                  (13, 144, 80, 16, 8, 90)])
def test_reach_rule_keeps_every_tile_where_alpha_reaches_threshold(seed, W, H, tw, th, rmax):
    """Every pixel centre of the rectangle where the FP64 splat has o G >= alpha_min (1 - 1e-5)
    lies in a kept tile; every kept tile is within 0.5 px (rows) and 0.011 px (columns) of the
    widened ellipse; kept tiles are a subset of the rectangle, and the rule drops tiles."""
    sp = random_splats(seed, 250, W, H, rmax, culled=0.0)
    keys, vals, _ = oracle.bin_instances(sp["uv"], sp["depth"], sp["radius"], W, H, tw, th,
                                         chol=sp["chol"], tau=sp["tau"])
    TX = -(-W // tw)
    kept = {}
    for k, i in zip((keys >> np.uint64(32)).astype(np.int64), vals):
        kept.setdefault(int(i), set()).add(int(k))
    total_rect = 0
    for i in range(len(sp["radius"])):
        x0, x1, y0, y1 = _rect_tiles(sp["uv"][i].astype(np.float64), int(sp["radius"][i]), W, H, tw, th)
        rect = {ty * TX + tx for ty in range(y0, y1) for tx in range(x0, x1)}
        total_rect += len(rect)
        mine = kept.get(i, set())
        assert mine <= rect
        if not rect:
            continue
        A, B, C = sp["conic"][i]
        u, v = sp["uv"][i].astype(np.float64)
        px = np.arange(x0 * tw, x1 * tw) + 0.5
        py = np.arange(y0 * th, y1 * th) + 0.5
        dx, dy = np.meshgrid(px - u, py - v)
        q = A * dx * dx + 2 * B * dx * dy + C * dy * dy
        alpha = sp["opacity"][i] * np.exp(-0.5 * q)
        hit = alpha >= ALPHA_MIN * (1 - 1e-5)
        ty_idx, tx_idx = np.nonzero(hit)
        need = {(y0 + r // th) * TX + (x0 + c // tw) for r, c in zip(ty_idx, tx_idx)}
        assert need <= mine, (i, sorted(need - mine))
        # tightness: some pixel column of the tile, moved by <= 0.011 px, meets the ellipse
        # q <= t at a y within the tile's band of pixel-centre rows
        t = float(sp["tau"][i]) * (1 + 2.0 ** -10) + 2.0 ** -10
        for tile in mine:
            tx, ty = tile % TX, tile // TX
            cx = np.arange(tx * tw, tx * tw + tw) + 0.5 - u
            cx = np.sign(cx) * np.maximum(np.abs(cx) - 0.011, 0.0)
            ya, yb = ty * th + 0.5 - v, ty * th + th - 0.5 - v
            ys = np.clip(-B * cx / C, ya, yb)
            qmin = (A * cx * cx + 2 * B * cx * ys + C * ys * ys).min()
            assert qmin <= t * (1 + 1e-5) + 1e-5, (i, tile, qmin, t)
    K = len(vals)
    assert K < 0.8 * total_rect, (K, total_rect)


def test_reach_rule_binning_is_the_rectangle_binning_filtered():
    """Same keys order as the rectangle binning with the dropped pairs removed (one stable sort
    of the emitted keys, ranges consistent)."""
    W, H, tw, th = 200, 120, 16, 16
    sp = random_splats(21, 400, W, H, 45, huge=2)
    k_r, v_r, r_r = oracle.bin_instances(sp["uv"], sp["depth"], sp["radius"], W, H, tw, th)
    k_e, v_e, r_e = oracle.bin_instances(sp["uv"], sp["depth"], sp["radius"], W, H, tw, th,
                                         chol=sp["chol"], tau=sp["tau"])
    pairs_e = list(zip(k_e.tolist(), v_e.tolist()))
    keep = set(pairs_e)
    filtered = [p for p in zip(k_r.tolist(), v_r.tolist()) if p in keep]
    assert filtered == pairs_e
    for t in range(r_e.shape[0]):
        a, b = r_e[t]
        assert np.all((k_e[a:b] >> np.uint64(32)) == t)
        assert (b - a) == int(np.sum((k_e >> np.uint64(32)) == t))
    # splats fainter than alpha_min reach no tile
    faint = sp["opacity"] < ALPHA_MIN
    assert faint.any() and not np.isin(np.nonzero(faint)[0], v_e).any()
    assert oracle.instance_count(sp["uv"], sp["radius"], W, H, tw, th, chol=sp["chol"], tau=sp["tau"]) == len(v_e)
