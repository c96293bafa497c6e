"""ctypes binding of include/kns.h: the same names, argument marshalling only.

Every function raises KnsError on a non-OK status.  Pointers are plain integers
(device addresses from torch tensors' data_ptr(), or host addresses).  Loading
fails loudly when libkns.so has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkns.so")

KNS_OK = 0
KNS_ERR_INVALID_ARG = 1
KNS_ERR_OUT_OF_MEMORY = 2
KNS_ERR_CUDA = 3
KNS_ERR_FORMAT = 4
KNS_ERR_UNSUPPORTED = 5
KNS_ERR_TIMEOUT = 6
KNS_ERR_BUSY = 7
KNS_ERR_INTERNAL = 8
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "FORMAT", 5: "UNSUPPORTED",
                6: "TIMEOUT", 7: "BUSY", 8: "INTERNAL"}
KNS_FP32 = 0
KNS_BF16 = 1


class KnsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("kns %s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


class kns_grid_desc(C.Structure):
    _fields_ = [("N", C.c_int32), ("pe_pos_L", C.c_int32), ("pe_dir_L", C.c_int32), ("sdf_hidden", C.c_int32),
                ("sdf_width", C.c_int32), ("feat_dim", C.c_int32), ("col_hidden", C.c_int32),
                ("col_width", C.c_int32), ("col_use_x", C.c_int32), ("occ_res", C.c_int32),
                ("softplus_beta", C.c_float), ("bbox_min", C.c_float * 3), ("bbox_max", C.c_float * 3)]


class kns_camera(C.Structure):
    _fields_ = [("c2w", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float)]


class kns_frame(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("normal", C.c_void_p), ("cell", C.c_void_p),
                ("steps", C.c_void_p), ("hit", C.c_void_p)]


class kns_view(C.Structure):
    _fields_ = [("cam", kns_camera), ("W", C.c_int32), ("H", C.c_int32), ("out", kns_frame), ("grid", C.c_int32),
                ("reserved", C.c_int32)]


class kns_train_batch(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("origins", C.c_void_p), ("dirs", C.c_void_p), ("target", C.c_void_p),
                ("n_strat", C.c_int32), ("n_imp", C.c_int32), ("u_strat", C.c_void_p), ("u_imp", C.c_void_p),
                ("n_eik", C.c_int64), ("eik_points", C.c_void_p), ("s", C.c_float), ("s_up", C.c_float),
                ("lambda_", C.c_float), ("h", C.c_float), ("t_fixed", C.c_void_p), ("timing", C.c_int32)]


class kns_train_stats(C.Structure):
    _fields_ = [("rays", C.c_int64), ("eik_points", C.c_int64), ("samples_per_ray", C.c_int32), ("pad", C.c_int32),
                ("records_coarse", C.c_int64), ("records_fd", C.c_int64), ("records_centre", C.c_int64),
                ("ms_coarse", C.c_float), ("ms_sort", C.c_float), ("ms_fd_forward", C.c_float),
                ("ms_centre_forward", C.c_float), ("ms_loss", C.c_float), ("ms_upstream", C.c_float),
                ("ms_centre_backward", C.c_float), ("ms_fd_backward", C.c_float), ("ms_total", C.c_float)]


class kns_pt_opts(C.Structure):
    _fields_ = [("spp", C.c_int32), ("max_depth", C.c_int32), ("seed", C.c_uint64), ("offset", C.c_float),
                ("horizon", C.c_float * 3), ("zenith", C.c_float * 3)]


class kns_render_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("eps_coarse", C.c_float), ("refine_steps", C.c_int32),
                ("inner_steps", C.c_int32), ("min_active", C.c_int32), ("tail_rays", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("static_tiles", C.c_int32), ("timing", C.c_int32),
                ("block_tiles", C.c_int32), ("bf16_inner_steps", C.c_int32), ("bf16_min_active", C.c_int32),
                ("bf16_rounds", C.c_int32)]


class kns_render_stats(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("rays", C.c_int64), ("hits", C.c_int64), ("samples_fp32", C.c_int64),
                ("samples_bf16", C.c_int64), ("ms_generate", C.c_float), ("ms_sort", C.c_float),
                ("ms_eval_fp32", C.c_float), ("ms_eval_bf16", C.c_float), ("ms_shade", C.c_float),
                ("ms_total", C.c_float), ("samples_tail", C.c_int64), ("refined", C.c_int64)]


class kns_peaks(C.Structure):
    _fields_ = [("ffma_flops", C.c_double), ("mufu_ops", C.c_double), ("sm_count", C.c_int32),
                ("sm_clock_khz", C.c_int32)]


class kns_round_info(C.Structure):
    _fields_ = [("live", C.c_int32), ("ms_sort", C.c_float), ("ms_eval_fp32", C.c_float), ("ms_eval_bf16", C.c_float),
                ("ms_advance", C.c_float), ("tiles", C.c_int32)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libkns.so (raises if it is missing: the product path has no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libkns.so is not built (run __graft_entry__.build() or "
                                  "python -m paper_2206_10885_gb300.build): %s" % LIB_PATH)
            L = C.CDLL(LIB_PATH)
            vp, st = C.c_void_p, C.c_int
            L.kns_create.argtypes = [C.c_int, C.POINTER(vp)]
            L.kns_create.restype = st
            L.kns_destroy.argtypes = [vp]
            L.kns_destroy.restype = None
            L.kns_last_error.argtypes = [vp]
            L.kns_last_error.restype = C.c_char_p
            L.kns_sync.argtypes = [vp, vp, C.c_int64]
            L.kns_sync.restype = st
            L.kns_load_grid.argtypes = [vp, C.POINTER(kns_grid_desc), vp, C.c_size_t, vp, C.POINTER(vp)]
            L.kns_load_grid.restype = st
            L.kns_load_grid_stack.argtypes = [vp, C.POINTER(kns_grid_desc), C.c_int32, vp, C.c_size_t, vp,
                                              C.POINTER(vp)]
            L.kns_load_grid_stack.restype = st
            L.kns_grid_stack_size.argtypes = [vp, C.POINTER(C.c_int32)]
            L.kns_grid_stack_size.restype = st
            L.kns_load_grid_file.argtypes = [vp, C.c_char_p, C.POINTER(vp)]
            L.kns_load_grid_file.restype = st
            L.kns_free_grid.argtypes = [vp]
            L.kns_free_grid.restype = None
            L.kns_grid_get_desc.argtypes = [vp, C.POINTER(kns_grid_desc)]
            L.kns_grid_get_desc.restype = st
            L.kns_copy_occupancy.argtypes = [vp, vp, vp, C.c_size_t]
            L.kns_copy_occupancy.restype = st
            L.kns_render.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                                     C.POINTER(kns_render_opts), C.POINTER(kns_frame), vp]
            L.kns_render.restype = st
            L.kns_sdf.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp, vp]
            L.kns_sdf.restype = st
            L.kns_render_noalloc.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                                             C.POINTER(kns_frame), vp]
            L.kns_render_noalloc.restype = st
            L.kns_render_views.argtypes = [vp, vp, C.POINTER(kns_view), C.c_int, C.c_int, C.c_float,
                                           C.POINTER(kns_render_opts), vp]
            L.kns_render_views.restype = st
            L.kns_get_render_stats.argtypes = [vp, C.POINTER(kns_render_stats)]
            L.kns_get_render_stats.restype = st
            L.kns_measure_peaks.argtypes = [vp, vp, C.POINTER(kns_peaks)]
            L.kns_measure_peaks.restype = st
            L.kns_selftest_timeout.argtypes = [vp, C.c_int32, vp]
            L.kns_selftest_timeout.restype = st
            L.kns_get_round_trace.argtypes = [vp, C.POINTER(kns_round_info), C.c_int32, C.POINTER(C.c_int32)]
            L.kns_get_round_trace.restype = st
            L.kns_trace_rays.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_int, C.c_float, C.POINTER(kns_frame),
                                         C.POINTER(kns_render_opts), vp]
            L.kns_trace_rays.restype = st
            L.kns_path_trace.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.POINTER(kns_pt_opts), C.c_int,
                                         C.c_float, vp, C.POINTER(kns_render_opts), vp]
            L.kns_path_trace.restype = st
            L.kns_train_forward.argtypes = [vp, C.POINTER(kns_grid_desc), vp, C.POINTER(kns_train_batch), vp, vp, vp,
                                            C.POINTER(C.c_uint64), vp]
            L.kns_train_forward.restype = st
            L.kns_train_backward.argtypes = [vp, C.c_uint64, vp, vp, vp]
            L.kns_train_backward.restype = st
            L.kns_train_step.argtypes = [vp, C.POINTER(kns_grid_desc), vp, C.POINTER(kns_train_batch), vp, vp, vp]
            L.kns_train_step.restype = st
            L.kns_train_get_stats.argtypes = [vp, C.POINTER(kns_train_stats)]
            L.kns_train_get_stats.restype = st
            _lib = L
    return _lib


def _check(status: int, ctx) -> None:
    if status != KNS_OK:
        msg = lib().kns_last_error(ctx)
        raise KnsError(status, msg.decode() if msg else "")


def kns_create(device: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().kns_create(device, C.byref(h)), None)
    return h.value


def kns_destroy(ctx: int) -> None:
    lib().kns_destroy(ctx)


def kns_last_error(ctx) -> str:
    m = lib().kns_last_error(ctx)
    return m.decode() if m else ""


def kns_sync(ctx: int, stream: int = 0, timeout_ms: int = -1) -> None:
    _check(lib().kns_sync(ctx, stream, timeout_ms), ctx)


def desc_struct(desc) -> kns_grid_desc:
    d = kns_grid_desc()
    for k in ("N", "pe_pos_L", "pe_dir_L", "sdf_hidden", "sdf_width", "feat_dim", "col_hidden", "col_width",
              "col_use_x", "occ_res"):
        setattr(d, k, int(getattr(desc, k)))
    d.softplus_beta = float(desc.softplus_beta)
    for a in range(3):
        d.bbox_min[a] = float(desc.bbox_min[a])
        d.bbox_max[a] = float(desc.bbox_max[a])
    return d


def kns_load_grid(ctx: int, desc, host_weights_ptr: int, n_floats: int, occ_words_ptr: int = None) -> int:
    h = C.c_void_p()
    d = desc_struct(desc)
    _check(lib().kns_load_grid(ctx, C.byref(d), host_weights_ptr, n_floats, occ_words_ptr, C.byref(h)), ctx)
    return h.value


def kns_load_grid_stack(ctx: int, desc, n_grids: int, host_weights_ptr: int, n_floats: int,
                        occ_words_ptr: int = None) -> int:
    h = C.c_void_p()
    d = desc_struct(desc)
    _check(lib().kns_load_grid_stack(ctx, C.byref(d), n_grids, host_weights_ptr, n_floats, occ_words_ptr,
                                     C.byref(h)), ctx)
    return h.value


def kns_grid_stack_size(grid: int) -> int:
    n = C.c_int32(0)
    _check(lib().kns_grid_stack_size(grid, C.byref(n)), None)
    return n.value


def kns_load_grid_file(ctx: int, path: str) -> int:
    h = C.c_void_p()
    _check(lib().kns_load_grid_file(ctx, path.encode(), C.byref(h)), ctx)
    return h.value


def kns_free_grid(grid: int) -> None:
    lib().kns_free_grid(grid)


def kns_grid_get_desc(grid: int) -> kns_grid_desc:
    d = kns_grid_desc()
    _check(lib().kns_grid_get_desc(grid, C.byref(d)), None)
    return d


def kns_copy_occupancy(ctx: int, grid: int, host_words_ptr: int, n_words: int) -> None:
    _check(lib().kns_copy_occupancy(ctx, grid, host_words_ptr, n_words), ctx)


def kns_render(ctx: int, grid: int, cams_host_ptr: int, n_cams: int, W: int, H: int, max_steps: int, eps: float,
               opts: kns_render_opts = None, frame: kns_frame = None, stream: int = 0) -> None:
    _check(lib().kns_render(ctx, grid, cams_host_ptr, n_cams, W, H, max_steps, eps,
                            C.byref(opts) if opts is not None else None,
                            C.byref(frame) if frame is not None else None, stream), ctx)


def kns_render_views(ctx: int, grid: int, views, max_steps: int, eps: float, opts: kns_render_opts = None,
                     stream: int = 0) -> None:
    """views: a ctypes array of kns_view (or a list, converted here)."""
    if not isinstance(views, C.Array):
        arr = (kns_view * max(1, len(views)))()
        for i, v in enumerate(views):
            arr[i] = v
        n = len(views)
        views = arr
    else:
        n = len(views)
    _check(lib().kns_render_views(ctx, grid, views, n, max_steps, eps,
                                  C.byref(opts) if opts is not None else None, stream), ctx)


def kns_get_render_stats(ctx: int) -> dict:
    st = kns_render_stats()
    _check(lib().kns_get_render_stats(ctx, C.byref(st)), ctx)
    return {k: getattr(st, k) for k, _ in kns_render_stats._fields_}


def kns_measure_peaks(ctx: int, stream: int = 0) -> dict:
    """Measured FP32 FMA FLOP/s and ex2 op/s of the context's device, its SM count and clock."""
    p = kns_peaks()
    _check(lib().kns_measure_peaks(ctx, stream, C.byref(p)), ctx)
    return {k: getattr(p, k) for k, _ in kns_peaks._fields_}


def kns_get_round_trace(ctx: int, max_rounds: int = 1024) -> list:
    """Per-round (live samples, sort / FP32 / BF16 evaluation ms) of the last render call."""
    buf = (kns_round_info * max_rounds)()
    n = C.c_int32(0)
    _check(lib().kns_get_round_trace(ctx, buf, max_rounds, C.byref(n)), ctx)
    return [{k: getattr(buf[i], k) for k, _ in kns_round_info._fields_} for i in range(min(n.value, max_rounds))]


def kns_selftest_timeout(ctx: int, which: int, stream: int = 0) -> None:
    """Runs a device wait that nothing satisfies (0: mbarrier, 1: grid barrier); the next sync reports it."""
    _check(lib().kns_selftest_timeout(ctx, which, stream), ctx)


def kns_sdf(ctx: int, grid: int, pts_ptr: int, n: int, sdf_ptr: int, feat_ptr: int = None, grad_ptr: int = None,
            stream: int = 0) -> None:
    _check(lib().kns_sdf(ctx, grid, pts_ptr, n, sdf_ptr, feat_ptr, grad_ptr, stream), ctx)


KNS_NOALLOC_MAX_RAYS = 262144
KNS_NOALLOC_MAX_CELLS = 32768
KNS_NOALLOC_MAX_CAMS = 64


def kns_render_noalloc(ctx: int, grid: int, cams_host_ptr: int, n_cams: int, W: int, H: int, max_steps: int,
                       eps: float, frame: kns_frame = None, stream: int = 0) -> None:
    _check(lib().kns_render_noalloc(ctx, grid, cams_host_ptr, n_cams, W, H, max_steps, eps,
                                    C.byref(frame) if frame is not None else None, stream), ctx)


def kns_train_forward(ctx: int, desc: kns_grid_desc, params_ptr: int, batch: kns_train_batch, loss_ptr: int,
                      rgb_ptr: int = None, t_ptr: int = None, stream: int = 0) -> int:
    tok = C.c_uint64(0)
    desc = desc_struct(desc)
    _check(lib().kns_train_forward(ctx, C.byref(desc), params_ptr, C.byref(batch), loss_ptr, rgb_ptr, t_ptr,
                                   C.byref(tok), stream), ctx)
    return tok.value


def kns_train_backward(ctx: int, token: int, dloss_ptr: int, grad_ptr: int, stream: int = 0) -> None:
    _check(lib().kns_train_backward(ctx, token, dloss_ptr, grad_ptr, stream), ctx)


def kns_train_step(ctx: int, desc: kns_grid_desc, params_ptr: int, batch: kns_train_batch, loss_ptr: int,
                   grad_ptr: int = None, stream: int = 0) -> None:
    desc = desc_struct(desc)
    _check(lib().kns_train_step(ctx, C.byref(desc), params_ptr, C.byref(batch), loss_ptr, grad_ptr, stream), ctx)


def kns_train_get_stats(ctx: int) -> dict:
    st = kns_train_stats()
    _check(lib().kns_train_get_stats(ctx, C.byref(st)), ctx)
    return {k: getattr(st, k) for k, _ in kns_train_stats._fields_ if k != "pad"}


def kns_trace_rays(ctx: int, grid: int, origins_ptr: int, dirs_ptr: int, n: int, max_steps: int, eps: float,
                   frame: kns_frame, opts: kns_render_opts = None, stream: int = 0) -> None:
    _check(lib().kns_trace_rays(ctx, grid, origins_ptr, dirs_ptr, n, max_steps, eps, C.byref(frame),
                                C.byref(opts) if opts is not None else None, stream), ctx)


def kns_path_trace(ctx: int, grid: int, cams_host_ptr: int, n_cams: int, W: int, H: int, pt: kns_pt_opts,
                   max_steps: int, eps: float, rgb_ptr: int, opts: kns_render_opts = None, stream: int = 0) -> None:
    _check(lib().kns_path_trace(ctx, grid, cams_host_ptr, n_cams, W, H, C.byref(pt), max_steps, eps, rgb_ptr,
                                C.byref(opts) if opts is not None else None, stream), ctx)
