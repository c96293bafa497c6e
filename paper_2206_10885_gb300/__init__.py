"""KiloNeuS sphere-tracing path for GB300: a thin Python layer over the C ABI (include/kns.h).

PyTorch is used only to own device memory and streams; every step of the path
runs in libkns.so's CUDA kernels.  The raw binding with the C names lives in
``_capi``; the helpers here allocate output tensors and marshal arguments.

    import paper_2206_10885_gb300 as kns
    from paper_2206_10885_gb300 import synth as S
    desc, w, cams, W, H, max_steps, eps = S.workload("c2")     # synthetic grid and cameras
    ctx = kns.Context(0)
    grid = kns.Grid.load(ctx, desc, w)                         # weights resident in HBM
    img = kns.render(ctx, grid, cams, W, H, max_steps, eps)    # dict of device tensors: rgb, depth,
                                                               # normal, cell, steps, hit
    d, z, g = kns.sdf(ctx, grid, points)                       # batch field query, points (n, 3) on cuda
    grid.free(); ctx.close()

kns.render_views (several views of one grid in one launch sequence), kns.trace_rays and
kns.path_trace (explicit rays, Lambertian bounces), kns.train (NeuS loss with the hand-written
backward as a torch.autograd.Function) and serve.RenderServer (continuous batching) build on the
same context and grid handles.
"""
from __future__ import annotations

import numpy as np

from . import _capi as capi
from . import train
from ._capi import KNS_BF16, KNS_FP32, KnsError

__all__ = ["capi", "KnsError", "KNS_FP32", "KNS_BF16", "Context", "Grid", "alloc_frame", "render", "sdf", "train",
           "trace_rays", "path_trace"]


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Context:
    """One kns_ctx on a CUDA device."""

    def __init__(self, device: int = 0):
        self.device = device
        self.handle = capi.kns_create(device)

    def sync(self, stream=None, timeout_ms: int = -1) -> None:
        capi.kns_sync(self.handle, _stream_ptr(stream), timeout_ms)

    def render_stats(self) -> dict:
        """Counters (and per-kernel-class device ms when rendered with tuning={'timing': 1}) of the last render."""
        return capi.kns_get_render_stats(self.handle)

    def measure_peaks(self, stream=None) -> dict:
        """FP32 FMA FLOP/s and ex2 op/s measured on the device by micro-kernels (roofline denominators)."""
        return capi.kns_measure_peaks(self.handle, _stream_ptr(stream))

    def round_trace(self) -> list:
        """Per-round live samples (and per-class device ms when rendered with tuning={'timing': 1}) of the
        last render call."""
        return capi.kns_get_round_trace(self.handle)

    def close(self) -> None:
        if self.handle:
            capi.kns_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Grid:
    """A resident Kilo-grid (weights and occupancy mask on the device)."""

    def __init__(self, ctx: Context, handle: int, desc):
        self.ctx, self.handle, self.desc = ctx, handle, desc

    @classmethod
    def load(cls, ctx: Context, desc, weights: np.ndarray, occ_words: np.ndarray = None) -> "Grid":
        w = np.ascontiguousarray(weights, dtype=np.float32)
        occ = None if occ_words is None else np.ascontiguousarray(occ_words, dtype=np.uint64)
        h = capi.kns_load_grid(ctx.handle, desc, w.ctypes.data, w.size, None if occ is None else occ.ctypes.data)
        return cls(ctx, h, desc)

    @classmethod
    def load_stack(cls, ctx: Context, desc, weights_list, occ_list=None) -> "Grid":
        """kns_load_grid_stack: several grids of one descriptor as one resident object; a view of
        render_views picks its grid by index (the request's optional fourth element)."""
        w = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float32).ravel() for x in weights_list]))
        occ = None
        if occ_list is not None:
            occ = np.ascontiguousarray(np.concatenate([np.asarray(o, dtype=np.uint64).ravel() for o in occ_list]))
        h = capi.kns_load_grid_stack(ctx.handle, desc, len(weights_list), w.ctypes.data, w.size,
                                     None if occ is None else occ.ctypes.data)
        return cls(ctx, h, desc)

    @property
    def n_grids(self) -> int:
        return capi.kns_grid_stack_size(self.handle)

    @classmethod
    def from_file(cls, ctx: Context, path: str) -> "Grid":
        h = capi.kns_load_grid_file(ctx.handle, path)
        return cls(ctx, h, capi.kns_grid_get_desc(h))

    def occupancy(self) -> np.ndarray:
        """The occupancy mask words (a stack: its grids' masks back to back)."""
        res = int(self.desc.occ_res)
        out = np.zeros(self.n_grids * ((res ** 3 + 63) // 64), dtype=np.uint64)
        capi.kns_copy_occupancy(self.ctx.handle, self.handle, out.ctypes.data, out.size)
        return out

    def free(self) -> None:
        if self.handle:
            capi.kns_free_grid(self.handle)
            self.handle = None


def alloc_frame(n_pix: int, device="cuda", extras: bool = True):
    """Output tensors of n_pix pixels plus the kns_frame that points at them."""
    import torch
    t = dict(rgb=torch.empty((n_pix, 3), dtype=torch.float32, device=device),
             depth=torch.empty(n_pix, dtype=torch.float32, device=device))
    if extras:
        t.update(normal=torch.empty((n_pix, 3), dtype=torch.float32, device=device),
                 cell=torch.empty(n_pix, dtype=torch.int32, device=device),
                 steps=torch.empty(n_pix, dtype=torch.int32, device=device),
                 hit=torch.empty(n_pix, dtype=torch.uint8, device=device))
    f = capi.kns_frame()
    for k in ("rgb", "depth", "normal", "cell", "steps", "hit"):
        setattr(f, k, t[k].data_ptr() if k in t else None)
    return t, f


TUNING_FIELDS = ("inner_steps", "min_active", "tail_rays", "blocks_per_sm", "static_tiles", "timing", "block_tiles",
                 "bf16_inner_steps", "bf16_min_active", "bf16_rounds")


def render_opts(precision: int = KNS_FP32, eps_coarse: float = 0.0, refine_steps: int = -1, tuning=None):
    o = capi.kns_render_opts()
    o.precision, o.eps_coarse, o.refine_steps = precision, eps_coarse, refine_steps
    for k, v in (tuning or {}).items():
        if k not in TUNING_FIELDS:
            raise KeyError(k)
        setattr(o, k, int(v))
    return o


def render(ctx: Context, grid: Grid, cams: np.ndarray, W: int, H: int, max_steps: int, eps: float,
           precision: int = KNS_FP32, out=None, stream=None, eps_coarse: float = 0.0, refine_steps: int = -1,
           tuning=None):
    """kns_render into fresh (or given) tensors; returns the dict of output tensors.

    tuning: optional dict of schedule knobs (see kns_render_opts); results do not depend on them.
    """
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    n_pix = cams.shape[0] * W * H
    if out is None:
        out = alloc_frame(n_pix, "cuda:%d" % ctx.device)
    t, f = out
    capi.kns_render(ctx.handle, grid.handle, cams.ctypes.data, cams.shape[0], W, H, max_steps, eps,
                    render_opts(precision, eps_coarse, refine_steps, tuning), f, _stream_ptr(stream))
    return t


def render_views(ctx: Context, grid: Grid, requests, max_steps: int, eps: float, precision: int = KNS_FP32,
                 stream=None, outs=None, tuning=None, eps_coarse: float = 0.0, refine_steps: int = -1):
    """kns_render_views: several (camera[16], W, H[, grid]) views in one launch sequence; grid picks the
    grid of a stack (Grid.load_stack; 0 when absent).

    Returns one dict of output tensors per request (allocated here unless `outs` gives them).
    """
    import ctypes as C
    if outs is None:
        outs = [alloc_frame(int(req[1]) * int(req[2]), "cuda:%d" % ctx.device) for req in requests]
    arr = (capi.kns_view * max(1, len(requests)))()
    for i, (req, (t, f)) in enumerate(zip(requests, outs)):
        cam, W, H = req[0], req[1], req[2]
        cam = np.ascontiguousarray(cam, dtype=np.float32).reshape(16)
        C.memmove(C.addressof(arr[i].cam), cam.ctypes.data, 64)
        arr[i].W, arr[i].H = int(W), int(H)
        arr[i].grid = int(req[3]) if len(req) > 3 else 0
        arr[i].out = f
    capi.kns_render_views(ctx.handle, grid.handle, arr if requests else [], max_steps, eps,
                          render_opts(precision, eps_coarse, refine_steps, tuning), _stream_ptr(stream))
    return [t for t, _ in outs]


def sdf(ctx: Context, grid: Grid, pts, want_feat: bool = True, want_grad: bool = True, stream=None):
    """kns_sdf on a (n, 3) float32 CUDA tensor; returns (d, feat, grad) tensors."""
    import torch
    pts = pts.contiguous()
    n = pts.shape[0]
    d = torch.empty(n, dtype=torch.float32, device=pts.device)
    feat = torch.empty((n, int(grid.desc.feat_dim)), dtype=torch.float32, device=pts.device) if want_feat else None
    grad = torch.empty((n, 3), dtype=torch.float32, device=pts.device) if want_grad else None
    capi.kns_sdf(ctx.handle, grid.handle, pts.data_ptr(), n, d.data_ptr(), feat.data_ptr() if want_feat else None,
                 grad.data_ptr() if want_grad else None, _stream_ptr(stream))
    return d, feat, grad


def trace_rays(ctx: Context, grid: Grid, origins, dirs, max_steps: int, eps: float, tuning=None, stream=None):
    """kns_trace_rays on (n, 3) float32 CUDA tensors; returns the dict of per-ray output tensors."""
    origins, dirs = origins.contiguous(), dirs.contiguous()
    n = origins.shape[0]
    t, f = alloc_frame(n, origins.device)
    capi.kns_trace_rays(ctx.handle, grid.handle, origins.data_ptr(), dirs.data_ptr(), n, max_steps, eps, f,
                        render_opts(KNS_FP32, tuning=tuning), _stream_ptr(stream))
    return t


SKY_HORIZON = (1.0, 1.0, 1.0)
SKY_ZENITH = (0.5, 0.7, 1.0)


def path_trace(ctx: Context, grid: Grid, cams: np.ndarray, W: int, H: int, spp: int = 16, max_depth: int = 4,
               seed: int = 0, offset: float = 1e-2, horizon=SKY_HORIZON, zenith=SKY_ZENITH, max_steps: int = 128,
               eps: float = 1e-4, tuning=None, stream=None):
    """kns_path_trace: Lambertian path-traced image as an (n_cams * H * W, 3) float32 CUDA tensor."""
    import torch
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    rgb = torch.empty((cams.shape[0] * W * H, 3), dtype=torch.float32, device="cuda:%d" % ctx.device)
    pt = capi.kns_pt_opts()
    pt.spp, pt.max_depth, pt.seed, pt.offset = spp, max_depth, seed, offset
    for k in range(3):
        pt.horizon[k] = horizon[k]
        pt.zenith[k] = zenith[k]
    capi.kns_path_trace(ctx.handle, grid.handle, cams.ctypes.data, cams.shape[0], W, H, pt, max_steps, eps,
                        rgb.data_ptr(), render_opts(KNS_FP32, tuning=tuning), _stream_ptr(stream))
    return rgb
