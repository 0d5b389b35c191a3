"""ctypes binding of the C ABI in include/gs.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and forwards its arguments
unchanged; the work happens in the sm_103a kernels of libgs_gb300.so.  Loading fails loudly
when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_float, c_void_p, c_uint32, c_uint64, c_size_t = (ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                                                          ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t)

GS_OK = 0
GS_ERR_INVALID_ARG = 1
GS_ERR_CAPACITY = 2
GS_ERR_TIMEOUT = 3
GS_ERR_CUDA = 4
GS_ERR_NUMERIC = 5
GS_ERR_INTERNAL = 6

GS_SORT_TWO_PHASE = 0
GS_SORT_KEY64 = 1
GS_STATIC_ORDER_MAX_N = 262144
GS_MAX_BATCH = 32
GS_TILES_REACH = 0
GS_TILES_RECT = 1

FLAG_CAPACITY = 1
FLAG_TIMEOUT = 2
FLAG_INTERNAL = 4
GS_DEFAULT_SPIN_LIMIT = 1 << 22


class gs_camera(ctypes.Structure):
    _fields_ = [("width", c_int), ("height", c_int), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("R", c_float * 9), ("t", c_float * 3), ("near_z", c_float)]


class gs_raster_config(ctypes.Structure):
    _fields_ = [("tile_w", c_int), ("tile_h", c_int), ("batch_depth", c_int), ("sort_mode", c_int),
                ("alpha_min", c_float), ("alpha_max", c_float), ("T_min", c_float), ("dilation", c_float),
                ("guard", c_float), ("extent", c_float), ("tile_rule", c_int), ("grad_limit", c_int),
                ("isotropic", c_int), ("spin_limit", ctypes.c_uint)]


class gs_gaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p), ("opacities", c_void_p),
                ("sh", c_void_p), ("n", c_int), ("sh_degree", c_int), ("sh_stride", c_int)]


class gs_gradients(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p), ("opacities", c_void_p),
                ("sh", c_void_p), ("mean2d", c_void_p)]


class gs_frame(ctypes.Structure):
    _fields_ = [("n", c_int), ("cam", gs_camera), ("cfg", gs_raster_config), ("capacity", c_uint64),
                ("ws", c_void_p), ("ws_bytes", c_size_t)]


class gs_layout(ctypes.Structure):
    _fields_ = [("xy", c_uint64), ("depth", c_uint64), ("conic_opacity", c_uint64), ("rgb", c_uint64),
                ("radius", c_uint64), ("tau", c_uint64), ("vals_sorted", c_uint64), ("keys_sorted", c_uint64), ("ranges", c_uint64),
                ("grad2d", c_uint64), ("status", c_uint64), ("total_bytes", c_uint64), ("tiles_x", c_int),
                ("tiles_y", c_int), ("key_passes", c_int), ("depth_passes", c_int), ("tile_order", c_uint64)]


class gs_device_status(ctypes.Structure):
    _fields_ = [("flags", c_uint32), ("num_instances", c_uint32), ("num_visible", c_uint32),
                ("num_nonfinite", c_uint32), ("blended_pairs", ctypes.c_uint64),
                ("num_segments", c_uint32), ("reserved", c_uint32)]


class gs_adam_group(ctypes.Structure):
    _fields_ = [("param", c_void_p), ("grad", c_void_p), ("m", c_void_p), ("v", c_void_p), ("activated", c_void_p),
                ("n", c_uint64), ("lr", c_float), ("activation", c_int)]


GS_ACT_NONE, GS_ACT_EXP, GS_ACT_SIGMOID = 0, 1, 2


class gs_param_arrays(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("logit_opacities", c_void_p),
                ("sh", c_void_p)]


class gs_density_config(ctypes.Structure):
    _fields_ = [("grad_threshold", c_float), ("min_opacity", c_float), ("split_scale", c_float),
                ("max_world_scale", c_float), ("max_screen_radius", c_float), ("split_factor", c_float)]

# (name, restype, argtypes) of every entry point declared in include/gs.h
SIGNATURES = [
    ("gs_default_config", None, [ctypes.POINTER(gs_raster_config)]),
    ("gs_workspace_size", c_size_t, [c_int, c_int, c_int, c_uint64, ctypes.POINTER(gs_raster_config)]),
    ("gs_workspace_layout", c_int, [c_int, c_int, c_int, c_uint64, ctypes.POINTER(gs_raster_config),
                                    ctypes.POINTER(gs_layout)]),
    ("gs_preprocess", c_int, [ctypes.POINTER(gs_frame), ctypes.POINTER(gs_gaussians), c_void_p]),
    ("gs_bin_sort", c_int, [ctypes.POINTER(gs_frame), c_void_p]),
    ("gs_render_forward", c_int, [ctypes.POINTER(gs_frame), ctypes.POINTER(c_float * 3), c_void_p, c_void_p,
                                  c_void_p, c_void_p]),
    ("gs_render_backward", c_int, [ctypes.POINTER(gs_frame), ctypes.POINTER(gs_gaussians),
                                   ctypes.POINTER(c_float * 3), c_void_p, c_void_p, c_void_p,
                                   ctypes.POINTER(gs_gradients), c_int, c_void_p]),
    ("gs_render_backward_tiles", c_int, [ctypes.POINTER(gs_frame), ctypes.POINTER(c_float * 3), c_void_p, c_void_p,
                                         c_void_p, c_void_p]),
    ("gs_render_backward_gaussians", c_int, [ctypes.POINTER(gs_frame), ctypes.POINTER(gs_gaussians),
                                             ctypes.POINTER(gs_gradients), c_int, c_void_p]),
    ("gs_read_status", c_int, [ctypes.POINTER(gs_frame), ctypes.POINTER(gs_device_status), c_void_p]),
    ("gs_batch_preprocess", c_int, [ctypes.POINTER(gs_frame), ctypes.POINTER(gs_gaussians), c_int, c_void_p]),
    ("gs_batch_bin_sort", c_int, [ctypes.POINTER(gs_frame), c_int, c_void_p]),
    ("gs_batch_render_forward", c_int, [ctypes.POINTER(gs_frame), c_int, ctypes.POINTER(c_float),
                                        ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                        c_void_p]),
    ("gs_batch_render_backward", c_int, [ctypes.POINTER(gs_frame), ctypes.POINTER(gs_gaussians), c_int,
                                         ctypes.POINTER(c_float), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                         ctypes.POINTER(c_void_p), ctypes.POINTER(gs_gradients), c_int, c_void_p]),
    ("gs_loss_workspace_size", c_size_t, [c_int, c_int]),
    ("gs_loss_l1_dssim", c_int, [c_void_p, c_void_p, c_int, c_int, c_float, c_void_p, c_size_t, c_void_p, c_void_p,
                                 c_void_p]),
    ("gs_adam_step", c_int, [ctypes.POINTER(gs_adam_group), c_int, c_float, c_float, c_float, c_int, c_void_p]),
    ("gs_density_stats", c_int, [ctypes.POINTER(gs_frame), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("gs_densify_scratch_size", c_size_t, [c_int]),
    ("gs_densify", c_int, [ctypes.POINTER(gs_density_config), c_int, c_int, ctypes.POINTER(gs_param_arrays),
                           ctypes.POINTER(gs_param_arrays), ctypes.POINTER(gs_param_arrays), c_void_p, c_void_p,
                           c_void_p, c_void_p, ctypes.POINTER(gs_param_arrays), ctypes.POINTER(gs_param_arrays),
                           ctypes.POINTER(gs_param_arrays), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                           c_void_p, c_void_p, c_size_t, c_void_p]),
    ("gs_opacity_reset", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_float, c_void_p]),
    ("gs_depth_order_static", c_int, [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("gs_status_string", ctypes.c_char_p, [c_int]),
    ("gs_bin_sort_timed", c_int, [ctypes.POINTER(gs_frame), ctypes.POINTER(c_float), ctypes.POINTER(ctypes.c_char_p),
                                  c_int, ctypes.POINTER(c_int), c_void_p]),
    ("gs_peak_fma", c_int, [c_int, c_int, c_void_p, c_void_p]),
    ("gs_peak_ex2", c_int, [c_int, c_int, c_void_p, c_void_p]),
    ("gs_peak_ops", ctypes.c_ulonglong, [c_int, c_int]),
]

_lib = None


def debug_build() -> bool:
    """GS_DEBUG=1 in the environment selects the bounds-checking build libgs_gb300_debug.so."""
    return os.environ.get("GS_DEBUG", "0") == "1"


def library_path() -> str:
    return _build.LIB_DEBUG if debug_build() else _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libgs_gb300.so (libgs_gb300_debug.so with GS_DEBUG=1).  Raises if it is missing
    (build it with __graft_entry__.build() or ``python -m paper_2308_04079_gb300.build``)."""
    global _lib
    if _lib is None:
        path = library_path()
        if build_if_missing and _build.needs_build(debug_build()):
            _build.build(debug=debug_build())
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA rasterizer library not built: {path} is missing")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class GSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (code {code})")


def status_string(code: int) -> str:
    return load().gs_status_string(code).decode()


def _check(code: int, where: str):
    if code != GS_OK:
        raise GSError(code, where)


def gs_default_config() -> gs_raster_config:
    cfg = gs_raster_config()
    load().gs_default_config(ctypes.byref(cfg))
    return cfg


def gs_workspace_size(n: int, width: int, height: int, capacity: int, cfg: gs_raster_config) -> int:
    return int(load().gs_workspace_size(n, width, height, capacity, ctypes.byref(cfg)))


def gs_workspace_layout(n: int, width: int, height: int, capacity: int, cfg: gs_raster_config) -> gs_layout:
    out = gs_layout()
    _check(load().gs_workspace_layout(n, width, height, capacity, ctypes.byref(cfg), ctypes.byref(out)),
           "gs_workspace_layout")
    return out


def gs_preprocess(frame: gs_frame, g: gs_gaussians, stream: int) -> None:
    _check(load().gs_preprocess(ctypes.byref(frame), ctypes.byref(g), stream), "gs_preprocess")


def gs_bin_sort(frame: gs_frame, stream: int) -> None:
    _check(load().gs_bin_sort(ctypes.byref(frame), stream), "gs_bin_sort")


def gs_render_forward(frame: gs_frame, bg, out_rgb: int, out_T: int, out_last: int, stream: int) -> None:
    b = (c_float * 3)(*[float(x) for x in bg])
    _check(load().gs_render_forward(ctypes.byref(frame), ctypes.byref(b), out_rgb, out_T, out_last, stream),
           "gs_render_forward")


def gs_render_backward(frame: gs_frame, g: gs_gaussians, bg, dL_drgb: int, T: int, last: int,
                       grads: gs_gradients, accumulate: bool, stream: int) -> None:
    b = (c_float * 3)(*[float(x) for x in bg])
    _check(load().gs_render_backward(ctypes.byref(frame), ctypes.byref(g), ctypes.byref(b), dL_drgb, T, last,
                                     ctypes.byref(grads), int(bool(accumulate)), stream), "gs_render_backward")


def gs_render_backward_tiles(frame: gs_frame, bg, dL_drgb: int, T: int, last: int, stream: int) -> None:
    b = (c_float * 3)(*[float(x) for x in bg])
    _check(load().gs_render_backward_tiles(ctypes.byref(frame), ctypes.byref(b), dL_drgb, T, last, stream),
           "gs_render_backward_tiles")


def gs_render_backward_gaussians(frame: gs_frame, g: gs_gaussians, grads: gs_gradients, accumulate: bool,
                                 stream: int) -> None:
    _check(load().gs_render_backward_gaussians(ctypes.byref(frame), ctypes.byref(g), ctypes.byref(grads),
                                               int(bool(accumulate)), stream), "gs_render_backward_gaussians")


def gs_read_status(frame: gs_frame, stream: int):
    st = gs_device_status()
    code = load().gs_read_status(ctypes.byref(frame), ctypes.byref(st), stream)
    if code in (GS_ERR_INVALID_ARG, GS_ERR_CUDA):
        raise GSError(code, "gs_read_status")
    return code, st


def gs_depth_order_static(n: int, depth: int, radius: int, order: int, status: int, stream: int) -> None:
    """Depth ordering with the library's static scratch (device pointers in, nothing
    allocated); see include/gs.h."""
    _check(load().gs_depth_order_static(n, depth, radius, order, status, stream), "gs_depth_order_static")


def gs_bin_sort_timed(frame: gs_frame, stream: int, cap: int = 32) -> list:
    """gs_bin_sort with every launch timed: [(label, ms), ...] in launch order (synchronises)."""
    ms = (c_float * cap)()
    names = (ctypes.c_char_p * cap)()
    count = c_int(0)
    _check(load().gs_bin_sort_timed(ctypes.byref(frame), ms, names, cap, ctypes.byref(count), stream),
           "gs_bin_sort_timed")
    return [(names[i].decode(), float(ms[i])) for i in range(count.value)]


def gs_peak_fma(blocks: int, iters: int, sink: int, stream: int) -> None:
    _check(load().gs_peak_fma(blocks, iters, sink, stream), "gs_peak_fma")


def gs_peak_ex2(blocks: int, iters: int, sink: int, stream: int) -> None:
    _check(load().gs_peak_ex2(blocks, iters, sink, stream), "gs_peak_ex2")


def gs_peak_ops(blocks: int, iters: int) -> int:
    return int(load().gs_peak_ops(blocks, iters))


def _ptrs(values):
    arr = (c_void_p * len(values))(*[int(v) for v in values])
    return ctypes.cast(arr, ctypes.POINTER(c_void_p)), arr


def gs_batch_preprocess(frames, gaussians, stream: int) -> None:
    fr = (gs_frame * len(frames))(*frames)
    gg = (gs_gaussians * len(gaussians))(*gaussians)
    _check(load().gs_batch_preprocess(fr, gg, len(frames), stream), "gs_batch_preprocess")


def gs_batch_bin_sort(frames, stream: int) -> None:
    fr = (gs_frame * len(frames))(*frames)
    _check(load().gs_batch_bin_sort(fr, len(frames), stream), "gs_batch_bin_sort")


def gs_batch_render_forward(frames, bg, out_rgb, out_T, out_last, stream: int) -> None:
    """bg: per-view (r, g, b); out_*: per-view device pointers."""
    fr = (gs_frame * len(frames))(*frames)
    b = (c_float * (3 * len(frames)))(*[float(x) for rgb in bg for x in rgb])
    p_rgb, k1 = _ptrs(out_rgb)
    p_T, k2 = _ptrs(out_T)
    p_last, k3 = _ptrs(out_last)
    _check(load().gs_batch_render_forward(fr, len(frames), b, p_rgb, p_T, p_last, stream), "gs_batch_render_forward")


def gs_batch_render_backward(frames, gaussians, bg, dL_drgb, T, last, grads, accumulate: bool, stream: int) -> None:
    fr = (gs_frame * len(frames))(*frames)
    gg = (gs_gaussians * len(gaussians))(*gaussians)
    gr = (gs_gradients * len(grads))(*grads)
    b = (c_float * (3 * len(frames)))(*[float(x) for rgb in bg for x in rgb])
    p_d, k1 = _ptrs(dL_drgb)
    p_T, k2 = _ptrs(T)
    p_last, k3 = _ptrs(last)
    _check(load().gs_batch_render_backward(fr, gg, len(frames), b, p_d, p_T, p_last, gr, int(bool(accumulate)),
                                           stream), "gs_batch_render_backward")


def gs_loss_workspace_size(width: int, height: int) -> int:
    return int(load().gs_loss_workspace_size(width, height))


def gs_loss_l1_dssim(img: int, target: int, width: int, height: int, lam: float, ws: int, ws_bytes: int,
                     out_loss: int, dL_dimg: int, stream: int) -> None:
    _check(load().gs_loss_l1_dssim(img, target, width, height, lam, ws, ws_bytes, out_loss, dL_dimg, stream),
           "gs_loss_l1_dssim")


def gs_adam_step(groups, beta1: float, beta2: float, eps: float, step: int, stream: int) -> None:
    arr = (gs_adam_group * len(groups))(*groups)
    _check(load().gs_adam_step(arr, len(groups), beta1, beta2, eps, step, stream), "gs_adam_step")


def gs_density_stats(frame, mean2d_grad: int, grad_accum: int, grad_count: int, max_radius: int | None,
                     stream: int) -> None:
    _check(load().gs_density_stats(ctypes.byref(frame), mean2d_grad, grad_accum, grad_count, max_radius, stream),
           "gs_density_stats")


def gs_densify_scratch_size(n: int) -> int:
    return int(load().gs_densify_scratch_size(n))


def gs_densify(cfg: gs_density_config, n: int, sh_floats: int, params: gs_param_arrays, adam_m: gs_param_arrays,
               adam_v: gs_param_arrays, grad_accum: int, grad_count: int, max_radius: int | None, normals: int,
               out_params: gs_param_arrays, out_m: gs_param_arrays, out_v: gs_param_arrays,
               out_grad_accum: int | None, out_grad_count: int | None, out_max_radius: int | None,
               out_scales: int | None, out_opacities: int | None, out_capacity: int, result: int, scratch: int,
               scratch_bytes: int, stream: int) -> None:
    _check(load().gs_densify(ctypes.byref(cfg), n, sh_floats, ctypes.byref(params), ctypes.byref(adam_m),
                             ctypes.byref(adam_v), grad_accum, grad_count, max_radius, normals,
                             ctypes.byref(out_params), ctypes.byref(out_m), ctypes.byref(out_v), out_grad_accum,
                             out_grad_count, out_max_radius, out_scales, out_opacities, out_capacity, result, scratch,
                             scratch_bytes, stream),
           "gs_densify")


def gs_opacity_reset(logit_opacities: int, adam_m: int | None, adam_v: int | None, opacities: int | None, n: int,
                     max_opacity: float, stream: int) -> None:
    _check(load().gs_opacity_reset(logit_opacities, adam_m, adam_v, opacities, n, max_opacity, stream),
           "gs_opacity_reset")
