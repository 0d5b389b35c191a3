"""gs_depth_order_static -- the depth ordering with its scratch in a static device array of
the library (nothing allocated per call) -- against the existing entry point gs_bin_sort.

On a frame of one 16x16 tile, binned with the paper's rectangle rule, every visible splat
covers the tile, so gs_bin_sort's sorted instance values are exactly the visible Gaussians in
(fp32 depth bits, index) order.  Two calls in a row with different inputs (and a different n)
check that every call re-initialises the shared scratch.  Kept in its own file, collected
last, and independent of the other tests' state."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _inputs(seed, n):
    rng = np.random.default_rng(seed)
    depth = rng.uniform(0.2, 30.0, n).astype(np.float32)
    depth[rng.random(n) < 0.1] = depth[0]                       # exact ties: order by index
    radius = rng.integers(1, 8, n).astype(np.int32)
    radius[rng.random(n) < 0.2] = 0                             # culled: after the visible ones
    return depth, radius


def _bin_sort_order(depth, radius):
    """Visible Gaussians in depth order from gs_bin_sort on a one-tile frame."""
    import torch
    from paper_2308_04079_gb300 import Frame, _abi, make_config
    n = depth.shape[0]
    cam = S.look_at_camera([0, 0, -4], [0, 0, 0], 16, 16, 60.0)
    fr = Frame(n, cam, make_config(tile=(16, 16), sort_mode="two_phase", tile_rule="rect"), capacity=n)
    xy = np.zeros((n, 4), np.float32)
    xy[:, :2] = 8.0                                             # every splat centred in the tile
    co = np.tile(np.array([1.0, 0.0, 1.0, 0.5], np.float32), (n, 1))
    fr.view("xy", torch.float32, 4 * n).copy_(torch.from_numpy(xy.reshape(-1)))
    fr.view("conic_opacity", torch.float32, 4 * n).copy_(torch.from_numpy(co.reshape(-1)))
    fr.view("tau", torch.float32, n).fill_(1.0)
    fr.view("depth", torch.float32, n).copy_(torch.from_numpy(depth))
    fr.view("radius", torch.int32, n).copy_(torch.from_numpy(radius))
    fr.bin_sort()
    code, st = fr.status()
    assert code == _abi.GS_OK
    K = int(st.num_instances)
    return fr.view("vals_sorted", torch.int32, max(K, 1)).cpu().numpy().view(np.uint32)[:K].copy()


def test_static_depth_order_matches_bin_sort_on_consecutive_calls():
    import torch
    from paper_2308_04079_gb300 import _abi
    nmax = _abi.GS_STATIC_ORDER_MAX_N
    order = torch.empty(nmax, dtype=torch.int32, device="cuda")
    status = torch.full((8,), -1, dtype=torch.int32, device="cuda")   # gs_device_status, 32 bytes
    stream = torch.cuda.current_stream().cuda_stream
    for seed, n in ((1, 200_000), (2, nmax), (3, 1_000)):
        depth, radius = _inputs(seed, n)
        d = torch.from_numpy(depth).cuda()
        r = torch.from_numpy(radius).cuda()
        _abi.gs_depth_order_static(n, d.data_ptr(), r.data_ptr(), order.data_ptr(), status.data_ptr(), stream)
        torch.cuda.synchronize()
        st = status.cpu().numpy().view(np.uint32)
        got = order[:n].cpu().numpy().view(np.uint32)
        ref = _bin_sort_order(depth, radius)
        K = ref.shape[0]
        assert st[0] == 0 and st[1] == 0 and st[2] == K and st[3] == 0
        assert np.array_equal(got[:K], ref)
        assert np.array_equal(got[K:], np.nonzero(radius <= 0)[0].astype(np.uint32))
        vis = np.nonzero(radius > 0)[0]
        assert np.array_equal(ref, vis[np.lexsort((vis, depth[vis].view(np.uint32)))].astype(np.uint32))


def test_static_depth_order_rejects_oversize_and_handles_empty():
    import torch
    from paper_2308_04079_gb300 import _abi
    nmax = _abi.GS_STATIC_ORDER_MAX_N
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    status = torch.full((8,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(_abi.GSError) as e:
        _abi.gs_depth_order_static(nmax + 1, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), status.data_ptr(), stream)
    assert e.value.code == _abi.GS_ERR_INVALID_ARG
    _abi.gs_depth_order_static(0, 0, 0, 0, status.data_ptr(), stream)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
