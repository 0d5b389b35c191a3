"""gs_bin_sort vs the oracle's binning definition (App. C, Algorithm 2), bit for bit:
instance count, sorted Gaussian indices, 64-bit keys (or tile ids) and tile ranges, for both
sort schedules, both tile rules (reachable tiles, the paper's 3-sigma rectangle), several
tile shapes, depth ties, culled, faint and off-screen splats, huge splats, empty input, and
instance counts spanning many sort tiles and scan chunks.  The screen-space inputs come from
the seeded generator, written straight into the workspace."""
import numpy as np
import pytest

import oracle
import synthetic as S
from screen_util import random_splats

pytestmark = pytest.mark.gpu


def _screen(seed, n, W, H, rmax, culled=0.1, ties=0.1, huge=0):
    return random_splats(seed, n, W, H, rmax, culled=culled, ties=ties, huge=huge)


def _oracle_bin(sp, W, H, tile, rule, capacity=None):
    kw = dict(chol=sp["chol"], tau=sp["tau"]) if rule == "reach" else {}
    return oracle.bin_instances(sp["uv"], sp["depth"], sp["radius"], W, H, tile[0], tile[1], capacity=capacity, **kw)


def _oracle_count(sp, W, H, tile=(16, 16), rule="reach"):
    kw = dict(chol=sp["chol"], tau=sp["tau"]) if rule == "reach" else {}
    return oracle.instance_count(sp["uv"], sp["radius"], W, H, tile[0], tile[1], **kw)


def _frame(sp, W, H, tile, mode, capacity, rule="reach"):
    """A frame whose workspace holds the screen-space splats sp, ready for gs_bin_sort."""
    import torch
    from paper_2308_04079_gb300 import Frame, make_config
    n = sp["uv"].shape[0]
    cam = S.look_at_camera([0, 0, -4], [0, 0, 0], W, H, 60.0)
    fr = Frame(n, cam, make_config(tile=tile, sort_mode=mode, tile_rule=rule), capacity=capacity)
    if n:
        xy4 = np.zeros((n, 4), np.float32)
        xy4[:, :2] = sp["uv"]                             # double-float mean with a zero low part
        co = np.zeros((n, 4), np.float32)
        co[:, :3] = sp["chol"]
        co[:, 3] = sp["opacity"]
        fr.view("xy", torch.float32, 4 * n).copy_(torch.from_numpy(xy4.reshape(-1)))
        fr.view("conic_opacity", torch.float32, 4 * n).copy_(torch.from_numpy(co.reshape(-1)))
        fr.view("tau", torch.float32, n).copy_(torch.from_numpy(sp["tau"]))
        fr.view("depth", torch.float32, n).copy_(torch.from_numpy(sp["depth"]))
        fr.view("radius", torch.int32, n).copy_(torch.from_numpy(sp["radius"]))
    return fr


def _expected_tile_order(ranges):
    """The render order gs_bin_sort must write: tiles by decreasing list-length class (four
    classes per power of two: the leading bit's position and the two bits below it; class 0
    for an empty tile), equal classes in increasing tile id."""
    length = (ranges[:, 1].astype(np.int64) - ranges[:, 0].astype(np.int64))
    cls = np.zeros(len(length), np.int64)
    for t, n in enumerate(length.tolist()):
        if n > 0:
            e = n.bit_length() - 1
            two = (n >> (e - 2)) & 3 if e >= 2 else (n << (2 - e)) & 3
            cls[t] = min(127, 1 + 4 * e + two)
    return np.argsort(-cls, kind="stable").astype(np.uint32)


def _check_tile_order(fr):
    import torch
    ranges = fr.view("ranges", torch.int32, 2 * fr.tiles).cpu().numpy().view(np.uint32).reshape(-1, 2)
    order = fr.view("tile_order", torch.int32, fr.tiles).cpu().numpy().view(np.uint32)
    assert np.array_equal(order, _expected_tile_order(ranges))


def _bin_gpu(sp, W, H, tile, mode, capacity, rule="reach"):
    fr = _frame(sp, W, H, tile, mode, capacity, rule)
    fr.bin_sort()
    code, st = fr.status()
    return fr, code, st


CASES = [
    (1, 3000, 200, 120, (16, 16), 30, 0),
    (2, 60000, 1920, 1080, (16, 16), 40, 3),
    (3, 20000, 640, 480, (8, 8), 25, 1),
    (4, 20000, 1000, 333, (16, 8), 25, 0),
    (5, 1, 64, 64, (16, 16), 10, 0),
    (6, 5000, 1920, 1080, (16, 16), 3, 0),
    # two-phase frames wider than 255 tiles keep the instance radix sort; taller than 256 tile
    # rows take two row passes; 255 columns fill every column digit but the padding one
    (7, 20000, 4400, 200, (16, 16), 20, 0),
    (8, 20000, 640, 4200, (16, 16), 20, 1),
    (9, 15000, 2040, 300, (8, 8), 12, 0),
    # large splats only (up to ~190 tile rows each): a segment-pass chunk of 256 entries spans
    # more than the 4096 rectangle rows it keeps in shared memory, so the rows past them are
    # evaluated again when their records are written
    (10, 600, 1920, 2400, (16, 16), 1500, 0),
]


@pytest.mark.parametrize("rule", ["reach", "rect"])
@pytest.mark.parametrize("mode", ["two_phase", "key64"])
@pytest.mark.parametrize("seed,n,W,H,tile,rmax,huge", CASES)
def test_bin_sort_bit_exact(mode, rule, seed, n, W, H, tile, rmax, huge):
    import torch
    from paper_2308_04079_gb300 import _abi
    sp = _screen(seed, n, W, H, rmax, huge=huge)
    keys_o, vals_o, ranges_o = _oracle_bin(sp, W, H, tile, rule)
    K = len(vals_o)
    fr, code, st = _bin_gpu(sp, W, H, tile, mode, capacity=K + 777, rule=rule)
    assert code == _abi.GS_OK
    assert st.num_instances == K
    vals = fr.view("vals_sorted", torch.int32, K).cpu().numpy().view(np.uint32)
    assert np.array_equal(vals, vals_o)
    ranges = fr.view("ranges", torch.int32, 2 * fr.tiles).cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert np.array_equal(ranges, ranges_o)
    _check_tile_order(fr)
    if mode == "key64":
        keys = fr.view("keys_sorted", torch.int64, K).cpu().numpy().view(np.uint64)
        assert np.array_equal(keys, keys_o)
    else:
        tiles = fr.view("keys_sorted", torch.int32, K).cpu().numpy().view(np.uint32)
        assert np.array_equal(tiles, (keys_o >> np.uint64(32)).astype(np.uint32))


@pytest.mark.parametrize("mode", ["two_phase", "key64"])
def test_bin_sort_empty_and_all_culled(mode):
    import torch
    from paper_2308_04079_gb300 import _abi
    fr, code, st = _bin_gpu(_screen(7, 0, 64, 48, 10), 64, 48, (16, 16), mode, 10)
    assert code == _abi.GS_OK and st.num_instances == 0
    assert np.all(fr.view("ranges", torch.int32, 2 * fr.tiles).cpu().numpy() == 0)
    sp = _screen(7, 500, 64, 48, 10)
    sp["radius"][:] = 0
    fr, code, st = _bin_gpu(sp, 64, 48, (16, 16), mode, 10)
    assert code == _abi.GS_OK and st.num_instances == 0
    # visible but fainter than alpha_min everywhere: no reachable tile
    sp = _screen(7, 500, 64, 48, 10, culled=0.0)
    sp["tau"][:] = -0.5
    fr, code, st = _bin_gpu(sp, 64, 48, (16, 16), mode, 10)
    assert code == _abi.GS_OK and st.num_instances == 0
    assert np.all(fr.view("ranges", torch.int32, 2 * fr.tiles).cpu().numpy() == 0)
    assert np.array_equal(fr.view("tile_order", torch.int32, fr.tiles).cpu().numpy(), np.arange(fr.tiles))


@pytest.mark.parametrize("mode", ["two_phase", "key64"])
def test_bin_sort_capacity_overflow_is_reported(mode):
    from paper_2308_04079_gb300 import _abi
    sp = _screen(8, 20000, 640, 480, 30)
    K = _oracle_count(sp, 640, 480)
    fr, code, st = _bin_gpu(sp, 640, 480, (16, 16), mode, K // 3)
    assert code == _abi.GS_ERR_CAPACITY
    assert st.num_instances == K
    # the workspace stays usable: a large enough frame bins the same input exactly
    fr2, code2, st2 = _bin_gpu(sp, 640, 480, (16, 16), mode, K)
    assert code2 == _abi.GS_OK and st2.num_instances == K


def test_bin_sort_deterministic_and_modes_agree():
    import torch
    sp = _screen(9, 40000, 1280, 720, 35, huge=2)
    K = _oracle_count(sp, 1280, 720)
    outs = []
    for mode in ("two_phase", "two_phase", "key64"):
        fr, code, st = _bin_gpu(sp, 1280, 720, (16, 16), mode, K)
        outs.append(fr.view("vals_sorted", torch.int32, K).cpu().numpy().copy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_batch_mixing_row_sort_and_radix_frames():
    """One gs_batch_bin_sort over frames that take the row-segmented tile sort (one or two row
    passes) and a frame wider than 255 tiles that takes the instance radix sort: every frame
    equals the oracle bit for bit."""
    import torch
    from paper_2308_04079_gb300 import FrameBatch, _abi
    shapes = [(640, 480, 30), (4400, 200, 20), (640, 4200, 20), (1920, 1080, 40)]
    sps, frames, refs = [], [], []
    for k, (W, H, rmax) in enumerate(shapes):
        sp = _screen(20 + k, 12000, W, H, rmax, huge=1)
        ref = _oracle_bin(sp, W, H, (16, 16), "reach")
        sps.append(sp)
        refs.append(ref)
        frames.append(_frame(sp, W, H, (16, 16), "two_phase", len(ref[1]) + 99))
    FrameBatch(frames, [None] * len(frames)).bin_sort()
    torch.cuda.synchronize()
    for fr, (keys_o, vals_o, ranges_o) in zip(frames, refs):
        code, st = fr.status()
        assert code == _abi.GS_OK
        K = len(vals_o)
        assert st.num_instances == K
        assert np.array_equal(fr.view("vals_sorted", torch.int32, K).cpu().numpy().view(np.uint32), vals_o)
        ranges = fr.view("ranges", torch.int32, 2 * fr.tiles).cpu().numpy().view(np.uint32).reshape(-1, 2)
        assert np.array_equal(ranges, ranges_o)
        tiles = fr.view("keys_sorted", torch.int32, K).cpu().numpy().view(np.uint32)
        assert np.array_equal(tiles, (keys_o >> np.uint64(32)).astype(np.uint32))
        _check_tile_order(fr)


def test_config3_full_frame_binning_bit_exact():
    """The benchmark frame (3M Gaussians, 1920x1080, two-phase schedule, reachable tiles, 16x16,
    the launch configuration bench.py times): its splats preprocessed on the GPU, then binned on
    the GPU and by the oracle's binning definition from the same fp32 screen-space values
    (screen mean without its low part): all 28M instances, their tile ids and every range equal,
    bit for bit."""
    import torch
    from paper_2308_04079_gb300 import Frame, GaussianTensors, _abi, make_config
    g, cam, _, _ = S.config3()
    gt = GaussianTensors.from_numpy(g, device="cuda").prepared()
    fr = Frame(gt.n, cam, make_config())
    fr.ensure_binned(gt)
    n = gt.n
    xy = fr.view("xy", torch.float32, 4 * n).reshape(n, 4)
    xy[:, 2:] = 0.0                                   # the oracle bins fp32 means
    fr.bin_sort()
    code, st = fr.status()
    assert code == _abi.GS_OK
    xy = xy.cpu().numpy()
    co = fr.view("conic_opacity", torch.float32, 4 * n).reshape(n, 4).cpu().numpy()
    tau = fr.view("tau", torch.float32, n).cpu().numpy()
    depth = fr.view("depth", torch.float32, n).cpu().numpy()
    radius = fr.view("radius", torch.int32, n).cpu().numpy()
    keys_o, vals_o, ranges_o = oracle.bin_instances(xy[:, :2], depth, radius, 1920, 1080, 16, 16,
                                                    chol=co[:, :3], tau=tau)
    K = len(vals_o)
    assert K > 20_000_000 and st.num_instances == K
    assert np.array_equal(fr.view("vals_sorted", torch.int32, K).cpu().numpy().view(np.uint32), vals_o)
    tiles = fr.view("keys_sorted", torch.int32, K).cpu().numpy().view(np.uint32)
    assert np.array_equal(tiles, (keys_o >> np.uint64(32)).astype(np.uint32))
    ranges = fr.view("ranges", torch.int32, 2 * fr.tiles).cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert np.array_equal(ranges, ranges_o)
    _check_tile_order(fr)


def test_config3_kept_tiles_cover_every_reaching_tile_and_stay_in_the_rectangle():
    """The benchmark frame (3M Gaussians, 1080p, reachable-tile rule, two-phase schedule) as
    bench.py bins it: every (Gaussian, tile) pair the GPU keeps lies in the Sec. 6 rectangle
    (under any rounding of it), and every pair of the FP64 brute-force set -- rectangle tiles in
    which some pixel centre certainly reaches alpha_min -- is kept.  This does not rely on the
    oracle's fp32 restatement of the reachable-tile rule."""
    import torch
    from gpu_util import REPORT
    from paper_2308_04079_gb300 import Frame, GaussianTensors, _abi, make_config
    g, cam, _, _ = S.config3()
    gt = GaussianTensors.from_numpy(g, device="cuda").prepared()
    fr = Frame(gt.n, cam, make_config())
    fr.ensure_binned(gt)
    code, st = fr.status()
    assert code == _abi.GS_OK
    K, T = int(st.num_instances), fr.tiles
    vals = fr.view("vals_sorted", torch.int32, K).cpu().numpy().astype(np.int64)
    ranges = fr.view("ranges", torch.int32, 2 * T).cpu().numpy().astype(np.int64).reshape(-1, 2)
    counts = ranges[:, 1] - ranges[:, 0]
    assert counts.sum() == K
    # the instances are sorted by tile id: tile t holds positions [start, end) in order
    nz = counts > 0
    assert np.all(np.diff(ranges[nz, 0]) > 0) and np.array_equal(ranges[nz, 0][1:], ranges[nz, 1][:-1])
    tile = np.repeat(np.arange(T, dtype=np.int64), counts)
    kept = np.sort(vals * T + tile)
    pp = oracle.preprocess(g, cam)
    TX = (cam.width + 15) // 16
    ro = pp["rect_out"][vals]
    tx, ty = tile % TX, tile // TX
    inside = (tx >= ro[:, 0]) & (tx < ro[:, 1]) & (ty >= ro[:, 2]) & (ty < ro[:, 3])
    assert inside.all(), int((~inside).sum())
    need = oracle.reach_needed(g, cam)
    missing = ~np.isin(need, kept, assume_unique=True)
    REPORT.append(f"binning config3: GPU keeps {K} (Gaussian, tile) pairs, all inside the rectangle; "
                  f"the FP64 brute-force set has {len(need)}, missing {int(missing.sum())}")
    assert len(need) > 0.9 * K and not missing.any(), need[missing][:10]
