"""Pins of the oracle's decision machinery (App. C numerical rules, Sec. 6 tile rectangle):
hand-built pixels placed exactly at, just off, and well away from each threshold -- the 1/255
skip, the 0.99 clamp, the 0.9999 stop, adjacent fp32 depth keys, the tile rectangle's radius
rounding, the colour clamp at 0 -- must or must not raise the decision, and the oracle's
flipped alternative must equal what the definition itself gives for the same scene moved to
the other side of the threshold (forward: colour, T, last Gaussian; backward: the allowance is
the gradient change that the flip really makes)."""
import math

import numpy as np
import pytest

import oracle
from synthetic import Gaussians, look_at_camera

Y00 = 0.5 / math.sqrt(math.pi)
AMIN = 1.0 / 255.0


def _gauss(means, scales, quats, opac, rgb):
    means = np.asarray(means, np.float64).reshape(-1, 3)
    n = means.shape[0]
    sh = (np.asarray(rgb, np.float64).reshape(n, 3) / Y00)[:, None, :]
    return Gaussians(means, np.asarray(scales, np.float64).reshape(n, 3), np.asarray(quats, np.float64).reshape(n, 4),
                     np.asarray(opac, np.float64).reshape(n), sh, 0)


def _axis_cam(width, height, distance=4.0):
    return look_at_camera([0.0, 0.0, -distance], [0.0, 0.0, 0.0], width, height, 60.0)


def _kinds(out, p):
    a = out["alt"]
    return sorted(int(k) for k in a["kind"][a["pix"] == p])


def _centre_splat(o, rgb=(0.8, 0.4, 0.2)):
    """One small isotropic splat centred on pixel (16, 16) of a 33x33 image (the principal
    point 16.5 is that pixel's centre, so G = 1 there and o G = o); its neighbours get
    G < 0.25, far from every threshold."""
    return _gauss([[0, 0, 0]], [[0.02] * 3], [[1, 0, 0, 0]], [o], [rgb]), _axis_cam(33, 33)


P16 = 16 * 33 + 16
BG = (0.1, 0.2, 0.3)


@pytest.mark.parametrize("delta", [1e-7, -1e-7])
def test_skip_near_threshold_is_flagged_and_its_alternative_is_the_other_side(delta):
    g, cam = _centre_splat(AMIN * (1 + delta))
    out = oracle.render_forward(g, cam, BG)
    assert _kinds(out, P16) == [oracle.DEC_SKIP]
    assert out["pix_dec"][16, 16] == 1 << (oracle.DEC_SKIP - 1)
    assert np.count_nonzero(out["pix_dec"]) == 1
    # the alternative is the definition evaluated just across the threshold
    other, _ = _centre_splat(AMIN * (1 - 3 * delta))
    ref = oracle.render_forward(other, cam, BG)
    a = out["alt"]
    assert len(a["pix"]) == 1
    np.testing.assert_allclose(a["img"][0], ref["img"][:, 16, 16], atol=1e-9)
    np.testing.assert_allclose(a["T"][0], ref["T"][16, 16], atol=1e-9)
    assert a["last_id"][0] == ref["last_id"][16, 16]
    assert (out["last_id"][16, 16] == 0) == (delta > 0) and (a["last_id"][0] == 0) == (delta < 0)


@pytest.mark.parametrize("delta", [1e-3, -1e-3, 0.5])
def test_skip_away_from_threshold_is_not_flagged(delta):
    g, cam = _centre_splat(AMIN * (1 + delta))
    out = oracle.render_forward(g, cam, BG)
    assert not out["pix_dec"].any() and len(out["alt"]["pix"]) == 0


@pytest.mark.parametrize("delta", [1e-7, -1e-7])
def test_clamp_near_threshold_is_flagged_with_its_derivative_switched(delta):
    g, cam = _centre_splat(0.99 * (1 + delta))
    out = oracle.render_forward(g, cam, BG)
    assert _kinds(out, P16) == [oracle.DEC_CLAMP]
    # the value is continuous across the clamp: the alternative differs by ~|delta|
    np.testing.assert_allclose(out["alt"]["img"][0], out["img"][:, 16, 16], atol=1e-6)
    # the gradient is not: unclamped, dL/do at the pixel is G (c - bg) . dL/dC; clamped, 0
    dimg = np.zeros((3, 33, 33))
    dimg[:, 16, 16] = (1.0, -0.5, 0.25)
    b = oracle.render_backward(g, cam, dimg, BG)
    want = abs(float(np.dot(np.array((0.8, 0.4, 0.2)) - BG, (1.0, -0.5, 0.25))))
    if delta > 0:       # clamped: no opacity gradient, the alternative has it
        assert b["opacities"][0] == 0.0
        assert b["allow"]["opacities"][0] == pytest.approx(want, rel=1e-6)
    else:
        assert b["opacities"][0] == pytest.approx(want, rel=1e-6)
        assert b["allow"]["opacities"][0] == pytest.approx(want, rel=1e-6)


@pytest.mark.parametrize("delta", [1e-2, -1e-2])
def test_clamp_away_from_threshold_is_not_flagged(delta):
    g, cam = _centre_splat(0.99 * (1 + delta))
    out = oracle.render_forward(g, cam, BG)
    assert not out["pix_dec"].any()


def _stop_stack(delta):
    """Three splats on pixel (16, 16), front to back o = 0.95, 0.95, o3 with
    0.05^2 (1 - o3) = 1e-4 (1 + delta): the third one's stop test sits at delta of 1e-4."""
    o3 = 1.0 - 0.04 * (1.0 + delta)
    means = [[0, 0, -1.0], [0, 0, -0.5], [0, 0, 0.0]]
    cols = [(0.9, 0.1, 0.1), (0.1, 0.9, 0.1), (0.1, 0.1, 0.9)]
    return _gauss(means, [[0.02] * 3] * 3, [[1, 0, 0, 0]] * 3, [0.95, 0.95, o3], cols), _axis_cam(33, 33)


@pytest.mark.parametrize("delta", [1e-6, -1e-6])
def test_stop_near_threshold_is_flagged_and_the_allowance_is_the_real_gradient_change(delta):
    g, cam = _stop_stack(delta)
    out = oracle.render_forward(g, cam, BG)
    assert _kinds(out, P16) == [oracle.DEC_STOP]
    blended = delta > 0            # T (1 - a) >= 1e-4: the third splat is blended
    assert out["last_id"][16, 16] == (2 if blended else 1)
    other, _ = _stop_stack(-delta)
    ref = oracle.render_forward(other, cam, BG)
    np.testing.assert_allclose(out["alt"]["img"][0], ref["img"][:, 16, 16], atol=1e-9)
    assert out["alt"]["last_id"][0] == ref["last_id"][16, 16]
    # backward: the flip changes the colour behind the two front splats and the third's own
    # terms; the allowance must equal the gradient change the flip really makes
    dimg = np.zeros((3, 33, 33))
    dimg[:, 16, 16] = (0.7, -1.1, 0.4)
    b = oracle.render_backward(g, cam, dimg, BG)
    r = oracle.render_backward(other, cam, dimg, BG)
    for k in ("opacities", "means", "sh"):
        change = np.abs(r[k] - b[k]).reshape(3, -1)
        np.testing.assert_allclose(b["allow"][k].reshape(3, -1), change, rtol=1e-4, atol=1e-9)
    assert np.all(b["allow"]["opacities"] > 1e-5)   # every splat of the pixel is affected


@pytest.mark.parametrize("delta", [5e-2, -5e-2])
def test_stop_away_from_threshold_is_not_flagged(delta):
    g, cam = _stop_stack(delta)
    out = oracle.render_forward(g, cam, BG)
    assert not out["pix_dec"].any()
    b = oracle.render_backward(g, cam, np.ones((3, 33, 33)), BG)
    assert all(not np.any(v) for v in b["allow"].values())


@pytest.mark.parametrize("ulps,flagged", [(0, True), (1, True), (2, False), (1000, False)])
def test_adjacent_depth_keys_are_flagged_and_the_alternative_swaps_them(ulps, flagged):
    """Two alpha = 0.5 splats on one pixel, camera-space depths 4 and 4 + ulps fp32 ulps
    (2^-21 each at 4): keys within one unit may swap under fp32 rounding of the depth."""
    cam = _axis_cam(33, 33)
    dz = ulps * 2.0 ** -21
    red, blue = (1.0, 0.0, 0.0), (0.0, 0.0, 1.0)
    g = _gauss([[0, 0, 0.0], [0, 0, dz]], [[0.02] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.5, 0.5], [red, blue])
    out = oracle.render_forward(g, cam)
    np.testing.assert_allclose(out["img"][:, 16, 16], [0.5, 0.0, 0.25], atol=1e-15)
    if not flagged:
        assert not out["pix_dec"].any()
        return
    assert _kinds(out, P16) == [oracle.DEC_SWAP]
    a = out["alt"]
    k = np.nonzero(a["pix"] == P16)[0][0]
    assert (a["g0"][k], a["g1"][k]) == (0, 1)
    np.testing.assert_allclose(a["img"][k], [0.25, 0.0, 0.5], atol=1e-15)
    assert a["last_id"][k] == 0


def _radius_splat(rr, o=0.95):
    """An isotropic splat on the optical axis of a 65x65 image (16x16 tiles), screen mean
    u = v = 32.5 (floor 32, well away from an integer), with 3 sqrt(lambda) = rr; r = ceil(rr)
    = 16 reaches tile column and row 3 (pixel 48 = floor(u) + r), r = 15 does not.  Pixel
    (48, 32) sees o G = o exp(-16^2 / (2 (rr/3)^2)) ~ 0.0057, well above 1/255."""
    cam = _axis_cam(65, 65)
    lam = (rr / 3.0) ** 2
    s = math.sqrt(lam - 0.3) * 4.0 / cam.fx
    return _gauss([[0, 0, 0]], [[s, s, s]], [[1, 0, 0, 0]], [o], [(0.5, 0.6, 0.7)]), cam


@pytest.mark.parametrize("rr,kind", [(15 * (1 + 1e-9), oracle.DEC_DROP), (15 * (1 - 1e-9), oracle.DEC_ADD)])
def test_tile_membership_near_the_radius_rounding_is_flagged(rr, kind):
    g, cam = _radius_splat(rr)
    pp = oracle.preprocess(g, cam)
    assert pp["amb"][0] & oracle.AMB_RECT
    assert pp["radius"][0] == (16 if kind == oracle.DEC_DROP else 15)
    out = oracle.render_forward(g, cam, BG)
    p = 32 * 65 + 48
    assert _kinds(out, p) == [kind]
    assert set(out["alt"]["kind"].tolist()) == {kind}
    # only tile column 3 and tile row 3 are uncertain, and only where the splat reaches 1/255
    py, px = np.nonzero(out["pix_dec"])
    assert np.all((px >= 48) | (py >= 48)) and np.all((px < 64) & (py < 64))
    # dropping it leaves the background, adding it gives the definition with r = 16
    other, _ = _radius_splat(15 * (1 + 1e-9) if kind == oracle.DEC_ADD else 15.5)
    with_it = oracle.render_forward(other, cam, BG)
    want = np.asarray(BG) if kind == oracle.DEC_DROP else with_it["img"][:, 32, 48]
    np.testing.assert_allclose(out["alt"]["img"][out["alt"]["pix"] == p][0], want, atol=1e-12)


def test_tile_membership_away_from_the_rounding_is_not_flagged():
    g, cam = _radius_splat(15.5)
    assert oracle.preprocess(g, cam)["amb"][0] == 0
    out = oracle.render_forward(g, cam, BG)
    assert not out["pix_dec"].any()


def _needle(opacity, W=129):
    """A splat on the optical axis, 30 px long and 0.6 px wide on screen (including the 0.3
    dilation), its long axis at 45 degrees; the pixel 35 columns and 35 rows from its centre
    lies on that axis, where the terms of the quadratic form cancel (Q >> |P|)."""
    cam = _axis_cam(W, W)
    sM = math.sqrt(30.0 ** 2 - 0.3) * 4.0 / cam.fx
    sm = math.sqrt(0.6 ** 2 - 0.3) * 4.0 / cam.fx
    c, s = math.cos(math.pi / 8), math.sin(math.pi / 8)     # 45 degrees about the view axis
    return _gauss([[0, 0, 0]], [[sM, sm, sm]], [[c, 0, 0, s]], [opacity], [(0.5, 0.5, 0.5)]), cam


def test_power_margin_follows_the_conditioning_of_the_quadratic_form():
    """Far along a needle's major axis an fp32 evaluation of the quadratic form loses digits to
    cancellation; the margin is eps_power times the magnitude sum Q of its terms, not |P|: a
    decision 1e-4 (relative) from the threshold is flagged there, although it is three times
    the plain alpha margin and far beyond eps_power |P|."""
    g, cam = _needle(0.01)
    pp = oracle.preprocess(g, cam)
    a, b, c = pp["conic"][0]
    dx = dy = 35.0
    P = 0.5 * (a * dx * dx + c * dy * dy) + b * dx * dy
    Q = 0.5 * (abs(a) * dx * dx + abs(c) * dy * dy) + abs(b * dx * dy)
    assert Q > 1000 * P
    eps = oracle.DEFAULT_CFG["eps_power"]
    assert eps * Q > 10 * 1e-4 > 10 * oracle.DEFAULT_CFG["eps_alpha"]
    p = (64 + 35) * 129 + 64 + 35
    for rel, flagged in ((1e-4, True), (-1e-4, True), (0.3, False)):
        gg, _ = _needle(AMIN * (1 + rel) * math.exp(P))
        out = oracle.render_forward(gg, cam, BG)
        assert (oracle.DEC_SKIP in _kinds(out, p)) == flagged, rel


def test_colour_clamp_near_zero_adds_that_channels_terms_to_the_allowance():
    """Degree-1 colour seen along the optical axis (Y_1^0 = sqrt(3 / (4 pi)) z, z = 1): the
    green channel's two terms cancel to 1e-9 of their size, so an fp32 sum may land on either
    side of the clamp at 0; the allowance of that Gaussian then holds the green channel's own
    chain-rule terms, Y_k |dL/dgreen| for every coefficient k, and nothing for red and blue."""
    cam = _axis_cam(33, 33)
    y10 = math.sqrt(3.0 / (4.0 * math.pi))
    sh = np.zeros((1, 4, 3))
    sh[0, 0] = np.array([0.5, 0.4, 0.3]) / Y00
    sh[0, 2, 1] = -0.4 / y10 * (1 - 1e-9)      # green: 0.4 - 0.4 (1 - 1e-9) = 4e-10
    g = Gaussians(np.zeros((1, 3)), np.full((1, 3), 0.1), np.array([[1.0, 0, 0, 0]]), np.array([0.7]), sh, 1)
    assert oracle.preprocess(g, cam)["amb"][0] & oracle.AMB_RGB
    dimg = np.zeros((3, 33, 33))
    dimg[:, 14:19, 14:19] = 1.0
    b = oracle.render_backward(g, cam, dimg, BG)
    al = b["allow"]["sh"][0]
    Y = np.array([Y00, 0.0, y10, 0.0])          # the basis along +z
    np.testing.assert_allclose(al[:, 1], Y * abs(b["rgb"][0, 1]), rtol=1e-12, atol=1e-300)
    assert al[0, 1] > 0 and not al[:, 0].any() and not al[:, 2].any()
    sh2 = sh.copy()
    sh2[0, 2, 1] = 0.0
    g2 = Gaussians(g.means, g.scales, g.quats, g.opacities, sh2, 1)
    assert not np.any(oracle.render_backward(g2, cam, dimg, BG)["allow"]["sh"])


def test_reach_needed_is_the_brute_force_set_of_tiles_reaching_alpha_min():
    """The (Gaussian, tile) pairs any binning must keep, against numpy brute force over every
    pixel of every certain rectangle tile from the oracle's own screen-space FP64 values."""
    from synthetic import tiny_scene
    g, cam = tiny_scene(61, n=150, width=70, height=45, deg=1, log_scale_mean=-2.2)
    cfg = oracle.cfg_array()
    got = oracle.reach_needed(g, cam, cfg)
    pp = oracle.preprocess(g, cam, cfg)
    TX = (cam.width + 15) // 16
    TY = (cam.height + 15) // 16
    want = []
    py, px = np.mgrid[0:cam.height, 0:cam.width]
    eps_a, eps_p = oracle.DEFAULT_CFG["eps_alpha"], oracle.DEFAULT_CFG["eps_power"]
    for i in range(g.n):
        if not pp["visible"][i] or pp["amb"][i] & oracle.AMB_CULL:
            continue
        a, b, c = pp["conic"][i]
        dx, dy = px + 0.5 - pp["uv"][i, 0], py + 0.5 - pp["uv"][i, 1]
        P = 0.5 * (a * dx * dx + c * dy * dy) + b * dx * dy
        Q = 0.5 * (abs(a) * dx * dx + abs(c) * dy * dy) + np.abs(b * dx * dy)
        hit = g.opacities[i] * np.exp(-P) >= AMIN * (1 + eps_a + eps_p * Q)
        x0, x1, y0, y1 = pp["rect_in"][i]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                if hit[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16].any():
                    want.append(i * TX * TY + ty * TX + tx)
    assert len(want) > 100
    np.testing.assert_array_equal(got, np.sort(np.array(want, np.int64)))
