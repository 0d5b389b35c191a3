"""Pins of the density-control oracle (Sec. 5.2, Algorithm 1) against definitions that do not
go through it: scipy's rotation for the split samples, closed forms for the statistics, the
logistic function for the pruning threshold, and hand-built decision cases."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import density as od


def _model(n, rng, sh_d=16):
    params = dict(means=rng.normal(size=(n, 3)), log_scales=rng.normal(-3, 1, size=(n, 3)),
                  quats=rng.normal(size=(n, 4)), logit_opacities=rng.normal(0, 2, size=n),
                  sh=rng.normal(size=(n, sh_d, 3)))
    m = {k: rng.normal(size=a.shape) for k, a in params.items()}
    v = {k: rng.uniform(0, 1, size=a.shape) for k, a in params.items()}
    return params, m, v


def _logit(p):
    return np.log(p / (1 - p))


def test_split_children_are_samples_of_the_parent_gaussian():
    """child = mu + R(q/|q|) diag(s) z with z the given draw: compared with scipy's rotation of
    the normalised quaternion (scalar last in scipy) and the parent's (pre-split) scales."""
    rng = np.random.default_rng(1)
    n = 40
    params, m, v = _model(n, rng)
    params["quats"] *= rng.uniform(0.3, 3.0, size=(n, 1))            # not unit length
    params["log_scales"] = rng.uniform(-1.0, 0.5, size=(n, 3))       # all above tau_S
    cfg = od.DensityConfig(split_scale=0.01, min_opacity=1e-9)
    acc, cnt, mr = np.ones(n), np.ones(n), np.zeros(n)
    z = rng.normal(size=(n, 2, 3))
    code, out, om, ov = od.densify(params, m, v, acc, cnt, mr, z, cfg)
    assert (code == od.SPLIT).all()
    assert out["means"].shape == (2 * n, 3)
    for i in range(n):
        q = params["quats"][i]
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        s = np.exp(params["log_scales"][i])
        for c in range(2):
            want = params["means"][i] + R @ (s * z[i, c])
            np.testing.assert_allclose(out["means"][2 * i + c], want, rtol=0, atol=1e-12)


def test_split_covariance_of_children_is_sigma():
    """Many children of one Gaussian: their sample covariance approaches R S^2 R^T (scipy)."""
    rng = np.random.default_rng(2)
    n = 4000
    q = np.array([0.8, -0.3, 0.5, 0.2])
    s = np.array([0.6, 0.15, 0.05])
    params, m, v = _model(n, rng)
    params["means"][:] = [1.0, -2.0, 0.5]
    params["quats"][:] = q
    params["log_scales"][:] = np.log(s)
    cfg = od.DensityConfig(split_scale=0.01, min_opacity=1e-9)
    z = rng.normal(size=(n, 2, 3))
    _, out, _, _ = od.densify(params, m, v, np.ones(n), np.ones(n), np.zeros(n), z, cfg)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]] / np.linalg.norm(q)).as_matrix()
    sigma = R @ np.diag(s * s) @ R.T
    d = out["means"] - [1.0, -2.0, 0.5]
    cov = d.T @ d / len(d)
    assert np.abs(cov - sigma).max() < 0.05 * s.max() ** 2
    # a transposed rotation would give R^T S^2 R, far from the samples
    assert np.abs(cov - R.T @ np.diag(s * s) @ R).max() > 0.1 * s.max() ** 2


def test_split_divides_scale_by_phi_and_copies_the_rest():
    rng = np.random.default_rng(3)
    n = 16
    params, m, v = _model(n, rng)
    params["log_scales"] = rng.uniform(-1.0, 0.0, size=(n, 3))
    cfg = od.DensityConfig(split_scale=0.01, min_opacity=1e-9)
    _, out, om, ov = od.densify(params, m, v, np.ones(n), np.ones(n), np.zeros(n), rng.normal(size=(n, 2, 3)), cfg)
    for i in range(n):
        for c in range(2):
            r = 2 * i + c
            np.testing.assert_allclose(np.exp(out["log_scales"][r]), np.exp(params["log_scales"][i]) / 1.6,
                                       rtol=1e-13)
            for k in ("quats", "logit_opacities", "sh"):
                assert np.array_equal(out[k][r], params[k][i])
            for k in od.PARAMS:
                assert not om[k][r].any() and not ov[k][r].any()


def test_clone_is_an_exact_copy_after_the_original():
    rng = np.random.default_rng(4)
    n = 12
    params, m, v = _model(n, rng)
    params["log_scales"] = rng.uniform(-9.0, -6.0, size=(n, 3))      # small: clone
    cfg = od.DensityConfig(split_scale=0.01, min_opacity=1e-9)
    code, out, om, ov = od.densify(params, m, v, np.ones(n), np.ones(n), np.zeros(n), np.zeros((n, 2, 3)), cfg)
    assert (code == od.CLONE).all()
    for i in range(n):
        for k in od.PARAMS:
            assert np.array_equal(out[k][2 * i], params[k][i]) and np.array_equal(out[k][2 * i + 1], params[k][i])
            assert np.array_equal(om[k][2 * i], m[k][i]) and np.array_equal(ov[k][2 * i], v[k][i])
            assert not om[k][2 * i + 1].any() and not ov[k][2 * i + 1].any()


def test_hand_built_decisions():
    """One row per rule, each next to its threshold (strict comparisons of Algorithm 1)."""
    cfg = od.DensityConfig(grad_threshold=0.0002, min_opacity=0.005, split_scale=0.03,
                           max_world_scale=0.5, max_screen_radius=20.0)
    rows = [  # (opacity, max scale, accum, count, max radius, expected)
        (0.004, 0.01, 1.0, 1, 0, od.PRUNE),        # transparent
        (0.006, 0.01, 0.0, 1, 0, od.KEEP),
        (0.5, 0.6, 0.0, 1, 0, od.PRUNE),           # too large in world space
        (0.5, 0.01, 0.0, 1, 21, od.PRUNE),         # too large on screen
        (0.5, 0.01, 0.0, 1, 20, od.KEEP),          # at the screen limit: kept
        (0.5, 0.01, 0.0004, 2, 0, od.KEEP),        # mean gradient equal to tau_pos: not above
        (0.5, 0.01, 0.0005, 2, 0, od.CLONE),
        (0.5, 0.04, 0.0005, 2, 0, od.SPLIT),
        (0.5, 0.04, 0.0005, 0, 0, od.KEEP),        # never seen: no mean gradient
        (0.004, 0.04, 1.0, 1, 0, od.PRUNE),        # pruning wins over densification
    ]
    n = len(rows)
    o = _logit(np.array([r[0] for r in rows]))
    ls = np.full((n, 3), np.log(1e-3))
    ls[:, 1] = np.log([r[1] for r in rows])
    acc = np.array([r[2] for r in rows], np.float32)
    cnt = np.array([r[3] for r in rows], np.float32)
    mr = np.array([r[4] for r in rows], np.float32)
    code = od.decide(o, ls, acc, cnt, mr, cfg)
    assert code.tolist() == [r[5] for r in rows]
    assert od.output_count(code) == 4 * 1 + 2 + 2


def test_prune_matches_logistic_definition_away_from_the_threshold():
    rng = np.random.default_rng(5)
    raw = rng.normal(-5.3, 0.5, size=20000)
    eps = 0.005
    alpha = 1 / (1 + np.exp(-raw))
    far = np.abs(alpha - eps) > 1e-6
    cfg = od.DensityConfig(min_opacity=eps)
    code = od.decide(raw, np.full((raw.size, 3), -9.0), np.zeros(raw.size), np.zeros(raw.size),
                     np.zeros(raw.size), cfg)
    assert np.array_equal((code == od.PRUNE)[far], (alpha < eps)[far])


def test_outputs_follow_source_order():
    rng = np.random.default_rng(6)
    n = 300
    params, m, v = _model(n, rng)
    params["means"][:, 0] = np.arange(n)              # tag rows by source index
    params["log_scales"] = rng.uniform(-5, -2, size=(n, 3))
    acc = rng.uniform(0, 0.001, size=n)
    cnt = rng.integers(0, 3, size=n).astype(np.float64)
    cfg = od.DensityConfig(split_scale=0.05)
    z = np.zeros((n, 2, 3))                          # children at the parent's mean
    code, out, _, _ = od.densify(params, m, v, acc, cnt, np.zeros(n), z, cfg)
    want = np.repeat(np.arange(n), [od.OUTPUTS[int(c)] for c in code])
    assert np.array_equal(out["means"][:, 0], want)
    offs = od.output_offsets(code)
    live = code != od.PRUNE
    assert np.array_equal(out["means"][offs[live], 0], np.arange(n)[live])
    assert len({int(c) for c in code}) == 4
    assert out["means"].shape[0] == od.output_count(code)


def test_empty_and_all_pruned():
    rng = np.random.default_rng(7)
    params, m, v = _model(0, rng)
    code, out, _, _ = od.densify(params, m, v, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros((0, 2, 3)),
                                 od.DensityConfig())
    assert code.size == 0 and out["sh"].shape == (0, 16, 3)
    params, m, v = _model(5, rng)
    params["logit_opacities"][:] = -20
    code, out, _, _ = od.densify(params, m, v, np.ones(5), np.ones(5), np.zeros(5), np.zeros((5, 2, 3)),
                                 od.DensityConfig())
    assert (code == od.PRUNE).all() and out["means"].shape == (0, 3)


def test_stats_closed_form():
    g = np.array([[1.0, 0.0], [0.0, 1.0], [3.0, 4.0], [5.0, 5.0]])
    r = np.array([3, 1, 2, 0])
    acc, cnt, mr = od.stats(g, r, 1920, 1080, np.zeros(4), np.zeros(4), np.full(4, 2.0))
    np.testing.assert_allclose(acc, [960.0, 540.0, np.hypot(3 * 960, 4 * 540), 0.0])
    assert cnt.tolist() == [1, 1, 1, 0]
    assert mr.tolist() == [3, 2, 2, 2]
    acc, cnt, mr = od.stats(g, r, 2, 2, acc, cnt, mr)
    np.testing.assert_allclose(acc[2], np.hypot(3 * 960, 4 * 540) + 5.0)
    assert cnt.tolist() == [2, 2, 2, 0]


def test_opacity_reset():
    raw = _logit(np.array([0.5, 0.02, 0.01, 0.005, 1e-5]))
    out, m, v = od.reset_opacity(raw, 0.01)
    alpha = 1 / (1 + np.exp(-out))
    assert (alpha <= 0.01 * (1 + 1e-6)).all()
    np.testing.assert_allclose(alpha[:3], 0.01, rtol=1e-6)
    np.testing.assert_allclose(out[3:], raw[3:], rtol=1e-6)
    assert not m.any() and not v.any()
