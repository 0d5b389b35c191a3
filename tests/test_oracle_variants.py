"""Pins of the oracle's ablation variants (Sec. 7.3): Limited-BW (gradients only for the N
front-most blended Gaussians of each pixel) and isotropic Gaussians (one scale, no rotation),
against finite differences of the forward definition, constructed depth orders and the
rotation invariance of s^2 I."""
import math
from types import SimpleNamespace

import numpy as np

import oracle
from synthetic import Gaussians, look_at_camera, tiny_scene

Y00 = 0.5 / math.sqrt(math.pi)


def _stack(n=4):
    """n wide Gaussians on the optical axis at depths 4, 4.3, 4.6, ... (front = index 0), each
    covering every pixel of a 6x6 image with alpha well above 1/255 and no stop."""
    rng = np.random.default_rng(3)
    means = np.zeros((n, 3))
    means[:, 2] = 0.3 * np.arange(n)
    means[:, :2] = rng.uniform(-0.2, 0.2, (n, 2))
    scales = rng.uniform(1.6, 2.4, (n, 3))
    quats = rng.normal(size=(n, 4))
    opac = rng.uniform(0.3, 0.5, n)
    sh = (rng.uniform(0.1, 0.9, (n, 3)) / Y00)[:, None, :]
    g = Gaussians(means, scales, quats, opac, sh, 0)
    cam = look_at_camera([0.0, 0.0, -4.0], [0.0, 0.0, 0.0], 6, 6, 60.0)
    return g, cam


def _loss(g, cam, dimg, bg, iso=False):
    f = oracle.render_forward_isotropic if iso else oracle.render_forward
    return float(np.sum(f(g, cam, bg)["img"] * dimg))


def _fd(g, cam, dimg, bg, name, idx, iso=False):
    arr = getattr(g, name)
    theta = float(arr[idx])
    h = 1e-6 * max(1.0, abs(theta))
    arr[idx] = theta + h
    lp = _loss(g, cam, dimg, bg, iso)
    arr[idx] = theta - h
    lm = _loss(g, cam, dimg, bg, iso)
    arr[idx] = theta
    return (lp - lm) / (2 * h)


def test_limited_bw_front_most_receive_the_full_gradient_the_rest_none():
    g, cam = _stack(4)
    bg = (0.2, 0.1, 0.3)
    dimg = np.random.default_rng(4).standard_normal((3, 6, 6))
    fwd = oracle.render_forward(g, cam, bg)
    assert (fwd["last"] == 4).all()                       # all four blended at every pixel
    lim = oracle.render_backward(g, cam, dimg, bg, oracle.cfg_array(grad_limit=2))
    for name in ("means", "scales", "quats", "opacities", "sh"):
        assert not lim[name][2:].any(), name               # the two back-most get nothing
    # the two front-most get the exact derivative of the full image (finite differences)
    for i in (0, 1):
        for name, idx in [("means", (i, 0)), ("means", (i, 2)), ("scales", (i, 1)), ("quats", (i, 3)),
                          ("opacities", (i,)), ("sh", (i, 0, 1))]:
            fd = _fd(g, cam, dimg, bg, name, idx)
            assert abs(lim[name][idx] - fd) <= 1e-5 * max(abs(fd), 1e-3), (name, idx, lim[name][idx], fd)


def test_limited_bw_n1_and_a_limit_beyond_the_depth():
    g, cam = _stack(5)
    bg = (0.0, 0.0, 0.0)
    dimg = np.random.default_rng(5).standard_normal((3, 6, 6))
    full = oracle.render_backward(g, cam, dimg, bg)
    one = oracle.render_backward(g, cam, dimg, bg, oracle.cfg_array(grad_limit=1))
    big = oracle.render_backward(g, cam, dimg, bg, oracle.cfg_array(grad_limit=100))
    for name in ("means", "scales", "quats", "opacities", "sh"):
        np.testing.assert_allclose(one[name][0], full[name][0], rtol=1e-12, atol=1e-15)
        assert not one[name][1:].any()
        np.testing.assert_allclose(big[name], full[name], rtol=1e-12, atol=1e-15)


def test_limited_bw_rank_follows_depth_not_index():
    """Reversing the index order of the stack keeps the gradient on the nearest Gaussians."""
    g, cam = _stack(4)
    rev = Gaussians(*(np.ascontiguousarray(a[::-1]) for a in (g.means, g.scales, g.quats, g.opacities, g.sh)), 0)
    dimg = np.random.default_rng(6).standard_normal((3, 6, 6))
    lim = oracle.render_backward(rev, cam, dimg, (0, 0, 0), oracle.cfg_array(grad_limit=2))
    assert not lim["opacities"][:2].any() and np.abs(lim["opacities"][2:]).min() > 0


def _iso_scene(seed=7, n=12):
    g, cam = tiny_scene(seed, n=n, width=20, height=16, deg=2, log_scale_mean=-1.8)
    s = np.exp(np.random.default_rng(seed).normal(-1.8, 0.3, n))
    iso = SimpleNamespace(means=np.array(g.means, np.float64), scales=s, quats=None,
                          opacities=np.array(g.opacities, np.float64), sh=np.array(g.sh, np.float64),
                          sh_degree=g.sh_degree)
    return iso, cam


def test_isotropic_image_is_rotation_invariant():
    """Sigma = R (s^2 I) R^T = s^2 I: the anisotropic renderer with scales (s, s, s) and any
    rotation draws the isotropic image."""
    iso, cam = _iso_scene()
    n = iso.means.shape[0]
    img = oracle.render_forward_isotropic(iso, cam)["img"]
    q = np.random.default_rng(8).normal(size=(n, 4))
    ani = Gaussians(iso.means, np.repeat(iso.scales[:, None], 3, 1), q, iso.opacities, iso.sh, iso.sh_degree)
    np.testing.assert_allclose(oracle.render_forward(ani, cam)["img"], img, rtol=0, atol=1e-12)
    assert img.std() > 1e-3


def test_isotropic_gradient_matches_finite_differences():
    iso, cam = _iso_scene()
    bg = (0.1, 0.2, 0.3)
    dimg = np.random.default_rng(9).standard_normal((3, cam.height, cam.width))
    ana = oracle.render_backward_isotropic(iso, cam, dimg, bg)
    assert "quats" not in ana and ana["scales"].shape == (iso.means.shape[0],)
    checked = 0
    for i in np.nonzero(np.abs(ana["opacities"]) > 0)[0][:6]:
        for name, idx in [("scales", (i,)), ("means", (i, 1)), ("opacities", (i,))]:
            fd = _fd(iso, cam, dimg, bg, name, idx, iso=True)
            assert abs(ana[name][idx] - fd) <= 1e-5 * max(abs(fd), 1e-3), (name, idx, ana[name][idx], fd)
            checked += 1
    assert checked >= 12
