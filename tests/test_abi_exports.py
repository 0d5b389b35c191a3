"""The C ABI library loads on a machine without a GPU, exports every entry point that
include/gs.h declares, and its host-only functions (configuration, workspace sizing and
layout, argument validation) behave as documented.  No kernel is launched here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2308_04079_gb300 import _abi, build
    build.build()
    build.build(debug=True)
    return _abi.load()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_four_stages():
    names = _declared_functions()
    for n in ("gs_preprocess", "gs_bin_sort", "gs_render_forward", "gs_render_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2308_04079_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gs_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing
    from paper_2308_04079_gb300 import _abi
    assert sorted(n for n, _, _ in _abi.SIGNATURES) == _declared_functions()
    # the GS_DEBUG build exports the same entry points
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB_DEBUG], capture_output=True, text=True,
                         check=True).stdout
    assert set(re.findall(r"\bT (gs_[a-z0-9_]+)$", out, flags=re.M)) >= set(_declared_functions())


def test_struct_layouts_match_header(lib, tmp_path):
    """ctypes mirrors of the ABI structs have the sizes the C compiler gives them."""
    from paper_2308_04079_gb300 import _abi
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "gs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(gs_camera), sizeof(gs_raster_config), sizeof(gs_gaussians),
         sizeof(gs_gradients), sizeof(gs_frame), sizeof(gs_layout), sizeof(gs_device_status),
         offsetof(gs_frame, capacity), offsetof(gs_frame, ws_bytes));
  return 0;
}'''
    src = str(tmp_path / "layout.c")
    exe = str(tmp_path / "layout")
    open(src, "w").write(code)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include", src, "-o", exe],
                   check=True)
    got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(_abi.gs_camera), ctypes.sizeof(_abi.gs_raster_config), ctypes.sizeof(_abi.gs_gaussians),
            ctypes.sizeof(_abi.gs_gradients), ctypes.sizeof(_abi.gs_frame), ctypes.sizeof(_abi.gs_layout),
            ctypes.sizeof(_abi.gs_device_status), _abi.gs_frame.capacity.offset, _abi.gs_frame.ws_bytes.offset]
    assert got == want


def test_default_config_is_the_papers(lib):
    from paper_2308_04079_gb300 import _abi
    c = _abi.gs_default_config()
    assert (c.tile_w, c.tile_h, c.batch_depth, c.sort_mode) == (16, 16, 128, _abi.GS_SORT_TWO_PHASE)
    assert c.alpha_min == pytest.approx(1 / 255) and c.alpha_max == pytest.approx(0.99)
    assert c.T_min == pytest.approx(1e-4) and c.dilation == pytest.approx(0.3)
    assert c.guard == pytest.approx(1.3) and c.extent == pytest.approx(3.0)
    assert c.spin_limit == _abi.GS_DEFAULT_SPIN_LIMIT == 1 << 22


def test_peak_microbenchmarks_validate_before_touching_the_device(lib):
    from paper_2308_04079_gb300 import _abi
    assert lib.gs_peak_fma(0, 10, 1, None) == _abi.GS_ERR_INVALID_ARG
    assert lib.gs_peak_ex2(4, 0, 1, None) == _abi.GS_ERR_INVALID_ARG
    assert lib.gs_peak_fma(4, 10, None, None) == _abi.GS_ERR_INVALID_ARG
    assert _abi.gs_peak_ops(304, 1000) == 304 * 1024 * 1000 * 16 * 8


def test_workspace_size_and_layout(lib):
    from paper_2308_04079_gb300 import _abi
    c = _abi.gs_default_config()
    s1 = _abi.gs_workspace_size(1000, 1920, 1080, 1 << 20, c)
    s2 = _abi.gs_workspace_size(1000, 1920, 1080, 1 << 21, c)
    assert 0 < s1 < s2
    L = _abi.gs_workspace_layout(1000, 1920, 1080, 1 << 20, c)
    assert L.total_bytes == s1
    assert (L.tiles_x, L.tiles_y) == (120, 68)
    assert L.key_passes == 2 and L.depth_passes == 4          # one row pass + the column pass
    offs = [L.xy, L.depth, L.conic_opacity, L.rgb, L.radius, L.vals_sorted, L.keys_sorted, L.ranges, L.grad2d,
            L.status]
    assert all(o % 16 == 0 for o in offs) and all(o < s1 for o in offs)
    c.sort_mode = _abi.GS_SORT_KEY64
    L64 = _abi.gs_workspace_layout(1000, 1920, 1080, 1 << 20, c)
    assert L64.key_passes == 6 and L64.depth_passes == 0       # 32 + 13 bits
    assert _abi.gs_workspace_size(0, 64, 64, 0, c) > 0         # empty scenes are valid


@pytest.mark.parametrize("W,H,tile,passes", [
    (1920, 1080, 16, 2),    # 120 x 68 tiles: row-segmented sort, one row pass + column pass
    (4080, 200, 16, 2),     # 255 tile columns: still the row sort
    (640, 4200, 16, 3),     # 263 tile rows: two row passes + column pass
    (4096, 200, 16, 2),     # 256 tile columns: instance radix sort, 3328 tiles -> 12 bits, 2 passes
    (4400, 4400, 16, 3),    # 275 x 275 tiles: radix sort, 17 bits -> 3 passes
    (2048, 2100, 8, 3),     # 256 x 263 tiles of 8 x 8: radix sort, 17 bits -> 3 passes
])
def test_tile_sort_schedule_passes(lib, W, H, tile, passes):
    """Two-phase frames up to 255 tile columns take the row-segmented tile sort (row byte
    passes over the segment records + one column pass), wider ones the byte passes over the
    instance tile ids; the sorted instances sit in the buffer the pass count selects."""
    from paper_2308_04079_gb300 import _abi
    c = _abi.gs_default_config()
    c.tile_w = c.tile_h = tile
    c.batch_depth = min(c.batch_depth, tile * tile)
    L = _abi.gs_workspace_layout(5000, W, H, 1 << 16, c)
    assert L.key_passes == passes and L.depth_passes == 4
    assert L.keys_sorted % 256 == 0 and L.vals_sorted % 256 == 0 and L.vals_sorted < L.total_bytes


@pytest.mark.parametrize("bad", [dict(tile_w=12), dict(batch_depth=0), dict(batch_depth=257), dict(sort_mode=7),
                                 dict(alpha_min=0.0), dict(alpha_max=1.5), dict(T_min=0.0)])
def test_invalid_config_rejected(lib, bad):
    from paper_2308_04079_gb300 import _abi
    c = _abi.gs_default_config()
    for k, v in bad.items():
        setattr(c, k, v)
    assert _abi.gs_workspace_size(10, 64, 64, 100, c) == 0
    with pytest.raises(_abi.GSError):
        _abi.gs_workspace_layout(10, 64, 64, 100, c)


def test_invalid_sizes_rejected(lib):
    from paper_2308_04079_gb300 import _abi
    c = _abi.gs_default_config()
    assert _abi.gs_workspace_size(-1, 64, 64, 100, c) == 0
    assert _abi.gs_workspace_size(10, 0, 64, 100, c) == 0
    assert _abi.gs_workspace_size(10, 64, 64, 1 << 31, c) == 0


def test_stage_calls_validate_before_touching_the_device(lib):
    """Null / undersized / misaligned descriptions return GS_ERR_INVALID_ARG synchronously."""
    from paper_2308_04079_gb300 import _abi
    L = _abi.load()
    assert L.gs_preprocess(None, None, None) == _abi.GS_ERR_INVALID_ARG
    assert L.gs_bin_sort(None, None) == _abi.GS_ERR_INVALID_ARG
    f = _abi.gs_frame()
    f.n = 10
    f.cam.width, f.cam.height, f.cam.fx, f.cam.fy, f.cam.near_z = 64, 64, 50.0, 50.0, 0.2
    f.cfg = _abi.gs_default_config()
    f.capacity = 100
    f.ws = 256
    f.ws_bytes = 16            # far too small
    assert L.gs_bin_sort(ctypes.byref(f), None) == _abi.GS_ERR_INVALID_ARG
    f.ws_bytes = _abi.gs_workspace_size(10, 64, 64, 100, f.cfg)
    f.ws = 257                 # misaligned
    assert L.gs_bin_sort(ctypes.byref(f), None) == _abi.GS_ERR_INVALID_ARG
    f.ws = 256
    g = _abi.gs_gaussians()
    g.n = 9                    # does not match the frame
    assert L.gs_preprocess(ctypes.byref(f), ctypes.byref(g), None) == _abi.GS_ERR_INVALID_ARG
    bg = (ctypes.c_float * 3)(0, 0, 0)
    assert L.gs_render_forward(ctypes.byref(f), ctypes.byref(bg), None, None, None, None) == _abi.GS_ERR_INVALID_ARG
    assert _abi.status_string(_abi.GS_ERR_CAPACITY) == "instance capacity exceeded"


def test_static_depth_order_validates_before_touching_the_device(lib):
    """The static-scratch depth ordering rejects n beyond its scratch, n < 0 and null pointers
    synchronously, without a device call."""
    from paper_2308_04079_gb300 import _abi
    L = _abi.load()
    nmax = _abi.GS_STATIC_ORDER_MAX_N
    assert L.gs_depth_order_static(nmax + 1, 256, 256, 256, 256, None) == _abi.GS_ERR_INVALID_ARG
    assert L.gs_depth_order_static(-1, 256, 256, 256, 256, None) == _abi.GS_ERR_INVALID_ARG
    assert L.gs_depth_order_static(10, 256, 256, 256, None, None) == _abi.GS_ERR_INVALID_ARG
    assert L.gs_depth_order_static(10, None, 256, 256, 256, None) == _abi.GS_ERR_INVALID_ARG
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    assert f"#define GS_STATIC_ORDER_MAX_N {nmax}" in src


def _fake_frames(count, width=64, height=64):
    from paper_2308_04079_gb300 import _abi
    frames = (_abi.gs_frame * count)()
    for f in frames:
        f.n = 10
        f.cam.width, f.cam.height, f.cam.fx, f.cam.fy, f.cam.near_z = width, height, 50.0, 50.0, 0.2
        f.cfg = _abi.gs_default_config()
        f.capacity = 100
        f.ws = 256
        f.ws_bytes = _abi.gs_workspace_size(10, width, height, 100, f.cfg)
    return frames


def test_batch_calls_validate_before_touching_the_device(lib):
    """Batches reject a view count outside [1, 32], frames with different tile shapes and
    gradient outputs shared between groups of frames, synchronously."""
    import ctypes as C
    from paper_2308_04079_gb300 import _abi
    L = _abi.load()
    frames = _fake_frames(2)
    assert L.gs_batch_bin_sort(frames, 0, None) == _abi.GS_ERR_INVALID_ARG
    big = _fake_frames(_abi.GS_MAX_BATCH + 1)
    assert L.gs_batch_bin_sort(big, _abi.GS_MAX_BATCH + 1, None) == _abi.GS_ERR_INVALID_ARG
    frames[1].cfg.tile_w, frames[1].cfg.tile_h = 8, 8
    frames[1].ws_bytes = _abi.gs_workspace_size(10, 64, 64, 100, frames[1].cfg)
    assert L.gs_batch_bin_sort(frames, 2, None) == _abi.GS_ERR_INVALID_ARG
    frames = _fake_frames(2)
    gs = (_abi.gs_gaussians * 2)()
    gr = (_abi.gs_gradients * 2)()
    for k in range(2):
        g = gs[k]
        g.n, g.sh_degree, g.sh_stride = 10, 3, 16
        base = 4096 * (k + 1)                      # two different scenes
        g.means, g.scales, g.quats, g.opacities, g.sh = base, base + 256, base + 512, base + 768, base + 1024
        r = gr[k]
        r.means, r.scales, r.quats, r.opacities, r.sh = 65536, 65536 + 256, 65536 + 512, 65536 + 768, 65536 + 1024
    bg = (C.c_float * 6)(*([0.0] * 6))
    ptrs = (C.c_void_p * 2)(256, 256)
    # different Gaussians writing the same gradient buffers
    code = L.gs_batch_render_backward(frames, gs, 2, bg, ptrs, ptrs, ptrs, gr, 0, None)
    assert code == _abi.GS_ERR_INVALID_ARG
