"""gs_preprocess vs the FP64 oracle: visibility, screen mean, depth, conic, radius, colour
(Sec. 4, Sec. 6, eq. volume-render, eq. quat)."""
import numpy as np
import pytest

import oracle
import synthetic as S
from gpu_util import REPORT, gpu_forward, screen_state

pytestmark = pytest.mark.gpu


def _cases():
    yield "tiny_deg3", S.tiny_scene(101, n=300, width=100, height=37)
    yield "tiny_deg1", S.tiny_scene(102, n=300, width=64, height=64, deg=1)
    g, cam, _ = S.config1()
    yield "config1", (g, cam)
    g, cam, _, _ = S.config2()
    yield "config2", (g, cam)


@pytest.mark.parametrize("name,scene", list(_cases()), ids=[c[0] for c in _cases()])
def test_preprocess_matches_oracle(name, scene):
    g, cam = scene
    run = gpu_forward(g, cam, (0.0, 0.0, 0.0))
    ss = screen_state(run)
    pp = oracle.preprocess(g, cam)
    amb = (pp["amb"] & (oracle.AMB_CULL | oracle.AMB_RECT)) != 0
    vis_g, vis_o = ss["radius"] > 0, pp["visible"] > 0
    assert np.array_equal(vis_g[~amb], vis_o[~amb])
    assert vis_o.sum() > 0.2 * len(vis_o)
    both = vis_g & vis_o
    uv = pp["uv"][both]
    # the screen mean is carried as a double-float: ~1e-9 px, far below fp32 rounding
    assert np.all(np.abs(ss["xy"][both] - uv) <= 1e-9 * np.maximum(1.0, np.abs(uv)))
    assert np.all(np.abs(ss["depth"][both] - pp["depth"][both]) <= 1e-6 * pp["depth"][both])
    con = pp["conic"][both]
    scale = np.maximum(np.abs(con[:, 0]), np.abs(con[:, 2]))[:, None]
    conic_err = float((np.abs(ss["conic"][both] - con) / scale).max())
    REPORT.append(f"preprocess {name}: conic relative error {conic_err:.2e}, "
                  f"depth {float((np.abs(ss['depth'][both] - pp['depth'][both]) / pp['depth'][both]).max()):.2e}")
    assert conic_err <= 1e-5
    sure = both & ~amb
    assert np.array_equal(ss["radius"][sure], pp["radius"][sure])
    assert np.all(np.abs(ss["rgb"][both] - pp["rgb"][both]) <= 2e-5)
    assert np.array_equal(ss["opacity"][both], g.opacities[both])


def test_nonfinite_inputs_are_culled_and_counted():
    from paper_2308_04079_gb300 import _abi
    g, cam = S.tiny_scene(103, n=64)
    g.means[3, 1] = np.nan
    g.scales[7, 0] = np.inf
    g.quats[11, 2] = np.nan
    g.opacities[13] = np.nan
    run = gpu_forward(g, cam, (0, 0, 0))
    ss = screen_state(run)
    assert all(ss["radius"][i] == 0 for i in (3, 7, 11, 13))
    code, st = run["frame"].status()
    assert code == _abi.GS_ERR_NUMERIC and st.num_nonfinite == 4
    assert np.all(np.isfinite(run["img"]))


def test_everything_behind_the_camera():
    g, cam = S.tiny_scene(104, n=50)
    g.means[:, 2] = -10.0        # behind the camera at z = -3
    run = gpu_forward(g, cam, (0.25, 0.5, 0.75))
    assert np.all(screen_state(run)["radius"] == 0)
    for ch, b in enumerate((0.25, 0.5, 0.75)):
        assert np.all(run["img"][ch] == np.float32(b))
    assert np.all(run["T"] == 1.0) and np.all(run["last"] == 0)
