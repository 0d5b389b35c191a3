"""Pins of the training-step oracle (Sec. 5.1): the loss L = 0.8 L1 + 0.2 (1 - SSIM) and its
gradient, and the Adam update, against facts that do not come from the oracle itself."""
import numpy as np
import pytest

from oracle import training as T


def _images(seed, H=19, W=23):
    rng = np.random.default_rng(seed)
    x = rng.random((3, H, W))
    y = np.clip(x + 0.2 * rng.standard_normal((3, H, W)), 0, 1)
    return x, y


def test_window_is_the_normalised_gaussian():
    w = T.window()
    assert w.shape == (11,) and abs(w.sum() - 1) < 1e-15
    assert np.allclose(w, w[::-1]) and np.argmax(w) == 5
    assert np.isclose(w[6] / w[5], np.exp(-1 / (2 * 1.5 ** 2)))


def test_window_sum_matches_scipy_correlate_with_zero_padding():
    scipy_ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    img = rng.random((17, 29))
    w2 = np.outer(T.window(), T.window())
    ref = scipy_ndimage.correlate(img, w2, mode="constant", cval=0.0)
    assert np.allclose(T.window_sum(img), ref, atol=1e-14)


def test_identical_images_have_zero_loss_and_zero_gradient():
    x, _ = _images(2)
    L, l1, ssim, g = T.loss(x, x)
    assert L == 0 and l1 == 0 and abs(ssim - 1) < 1e-12
    assert np.abs(g).max() < 1e-12


def test_constant_images_interior_ssim_closed_form():
    """Two constant images a, b: away from the zero-padded border every window sees constants,
    so the variances vanish and SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.3, 0.7
    x = np.full((3, 30, 30), a)
    y = np.full((3, 30, 30), b)
    s = T.ssim_map(x, y)
    interior = s[:, 5:-5, 5:-5]
    assert np.allclose(interior, (2 * a * b + T.C1) / (a * a + b * b + T.C1), atol=1e-13)


def test_loss_is_the_weighted_sum_of_its_terms():
    x, y = _images(3)
    L, l1, ssim, _ = T.loss(x, y, lam=0.2)
    assert np.isclose(l1, np.abs(x - y).mean())
    assert np.isclose(ssim, T.ssim_map(x, y).mean())
    assert np.isclose(L, 0.8 * l1 + 0.2 * (1 - ssim))


def test_loss_gradient_matches_central_differences():
    x, y = _images(4, H=13, W=15)
    lam = 0.2
    _, _, _, g = T.loss(x, y, lam)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(60):
        c, i, j = rng.integers(0, 3), rng.integers(0, 13), rng.integers(0, 15)
        if abs(x[c, i, j] - y[c, i, j]) < 1e-4:
            continue   # |x - y| is not differentiable there
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (T.loss(xp, y, lam)[0] - T.loss(xm, y, lam)[0]) / (2 * h)
        assert abs(fd - g[c, i, j]) <= 1e-7 * max(1.0, abs(fd)) + 1e-10, (c, i, j, fd, g[c, i, j])


def test_ssim_gradient_alone_matches_central_differences():
    """lambda = 1: the SSIM part only (its coefficient-map chain rule in isolation)."""
    x, y = _images(6, H=12, W=12)
    _, _, _, g = T.loss(x, y, lam=1.0)
    h = 1e-6
    for (c, i, j) in [(0, 0, 0), (1, 5, 7), (2, 11, 11), (0, 6, 0), (1, 0, 9)]:
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (T.loss(xp, y, 1.0)[0] - T.loss(xm, y, 1.0)[0]) / (2 * h)
        assert abs(fd - g[c, i, j]) <= 1e-7 * max(1.0, abs(fd)) + 1e-11


def test_adam_first_step_closed_form():
    """Step 1 with zero moments: the bias-corrected update is lr g / (|g| + eps)."""
    rng = np.random.default_rng(7)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, eps = 0.01, 1e-8
    p1, m1, v1, _ = T.adam_step(p, g, np.zeros(50), np.zeros(50), lr, 1, eps=eps)
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_adam_activation_chain_rules_match_finite_differences():
    """The raw gradient is the activated-value gradient times act'(raw): checked by a
    central difference of the activation."""
    rng = np.random.default_rng(8)
    raw = rng.standard_normal(20)
    g = rng.standard_normal(20)
    h = 1e-6
    for act in ("exp", "sigmoid"):
        dact = (T.activate(raw + h, act) - T.activate(raw - h, act)) / (2 * h)
        # with b1 = b2 = 0 and step 1 the update is lr * g_raw / (|g_raw| + eps): recover g_raw's sign
        p1, m1, _, _ = T.adam_step(raw, g, np.zeros(20), np.zeros(20), 1.0, 1, act, b1=0.0, b2=0.0)
        assert np.allclose(m1, g * dact, rtol=1e-8)


def test_adam_converges_on_a_quadratic():
    """Minimising 0.5 |p - p*|^2 drives p to p* (a behavioural check of the update's sign and
    scale)."""
    rng = np.random.default_rng(9)
    target = rng.standard_normal(10)
    p = np.zeros(10)
    m = np.zeros(10)
    v = np.zeros(10)
    for t in range(1, 3001):
        p, m, v, _ = T.adam_step(p, p - target, m, v, 0.01, t, eps=1e-8)
    assert np.abs(p - target).max() < 1e-3


def test_position_learning_rate_decays_exponentially():
    lr = [T.position_lr(s, 1.6e-4, 1.6e-6, 30000) for s in (0, 15000, 30000, 40000)]
    assert np.isclose(lr[0], 1.6e-4) and np.isclose(lr[2], 1.6e-6) and np.isclose(lr[3], 1.6e-6)
    assert np.isclose(lr[1], np.sqrt(1.6e-4 * 1.6e-6))
