"""FP64 oracle of the KiloNeuS sphere-tracing path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``kns_oracle.c`` (plain C, FP64,
OpenMP over rays), which shares no code with the CUDA library.  Descriptors are
duck-typed: any object with the grid fields (N, pe_pos_L, ..., bbox_max) works,
so this package imports nothing from the product package.

Every function here follows the paper's definitions; the C file's header lists
which section or equation each step restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kns_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Desc(C.Structure):
    _fields_ = [("N", C.c_int32), ("pe_pos_L", C.c_int32), ("pe_dir_L", C.c_int32),
                ("sdf_hidden", C.c_int32), ("sdf_width", C.c_int32), ("feat_dim", C.c_int32),
                ("col_hidden", C.c_int32), ("col_width", C.c_int32), ("col_use_x", C.c_int32),
                ("occ_res", C.c_int32), ("beta", C.c_double), ("bmin", C.c_double * 3),
                ("bmax", C.c_double * 3)]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, -O2, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            d = C.POINTER(C.c_double)
            f = C.POINTER(C.c_float)
            i32 = C.POINTER(C.c_int32)
            i64 = C.POINTER(C.c_int64)
            u8 = C.POINTER(C.c_uint8)
            u64 = C.POINTER(C.c_uint64)
            D = C.POINTER(_Desc)
            L.ko_params_cell.restype = C.c_int64
            L.ko_params_cell.argtypes = [D]
            L.ko_params_sdf.restype = C.c_int64
            L.ko_params_sdf.argtypes = [D]
            L.ko_pe.argtypes = [C.c_int, C.c_int, d, d]
            L.ko_softplus.restype = C.c_double
            L.ko_softplus.argtypes = [C.c_double, C.c_double]
            L.ko_cell.restype = C.c_int
            L.ko_cell.argtypes = [D, d]
            L.ko_sdf_eval.restype = C.c_double
            L.ko_sdf_eval.argtypes = [D, f, C.c_int, d, d, d]
            L.ko_colour_eval.argtypes = [D, f, C.c_int, d, d, d, d, d]
            L.ko_sdf_batch.argtypes = [D, f, C.c_int64, d, d, d, d, i32]
            L.ko_occupancy.argtypes = [D, f, C.c_int, C.c_double, u64]
            L.ko_ray.argtypes = [f, C.c_int, C.c_int, d, d]
            L.ko_render.argtypes = [D, f, u64, f, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.c_int64, i64, f, f, f, i32, u8, i32, d, u8]
            L.ko_trace_rays.argtypes = [D, f, u64, C.c_int64, d, d, C.c_int, C.c_double, d, i32, i32, d, d]
            L.ko_march_roots.argtypes = [D, f, C.c_int64, d, d, d, d, C.c_double, C.c_double, d]
            L.ko_first_occupied.restype = C.c_int
            L.ko_first_occupied.argtypes = [D, u64, d, d, C.c_double, d, i32]
            L.ko_train_loss.restype = C.c_double
            L.ko_train_loss.argtypes = [D, f, C.c_double, C.c_double, C.c_int64, d, d, d, C.c_int, d, C.c_int, d,
                                        C.c_int64, d, C.c_double, C.c_double, d, d, d, d]
            L.ko_train_grad.restype = C.c_double
            L.ko_train_grad.argtypes = L.ko_train_loss.argtypes[:-1]
            L.ko_splitmix64.restype = C.c_uint64
            L.ko_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
            L.ko_pt_uniform.restype = C.c_double
            L.ko_pt_uniform.argtypes = [C.c_uint64, C.c_int64, C.c_int, C.c_int]
            L.ko_cosine_dir.argtypes = [d, C.c_double, C.c_double, d]
            L.ko_sky.argtypes = [d, d, d, d]
            L.ko_path_trace.argtypes = [D, f, u64, f, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_double, C.c_double, C.c_uint64, d, d, C.c_int64, i64, d, d, i32]
            L.ko_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _desc(g) -> _Desc:
    s = _Desc()
    for k in ("N", "pe_pos_L", "pe_dir_L", "sdf_hidden", "sdf_width", "feat_dim", "col_hidden",
              "col_width", "col_use_x", "occ_res"):
        setattr(s, k, int(getattr(g, k)))
    s.beta = float(g.softplus_beta)
    for a in range(3):
        s.bmin[a] = float(g.bbox_min[a])
        s.bmax[a] = float(g.bbox_max[a])
    return s


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def _f32(w):
    return np.ascontiguousarray(w, dtype=np.float32)


def num_threads() -> int:
    return lib().ko_num_threads()


def params_per_cell(g) -> int:
    return lib().ko_params_cell(C.byref(_desc(g)))


def params_sdf(g) -> int:
    return lib().ko_params_sdf(C.byref(_desc(g)))


def pe(L: int, p) -> np.ndarray:
    """gamma_L(p) of Eq. 1 (raw coordinates first)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(p.size * (1 + 2 * L))
    lib().ko_pe(L, p.size, _p(p, C.c_double), _p(out, C.c_double))
    return out


def softplus(s: float, beta: float) -> float:
    return lib().ko_softplus(float(s), float(beta))


def cell(g, x) -> int:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().ko_cell(C.byref(_desc(g)), _p(x, C.c_double))


def sdf_cell(g, w, cell_id: int, x, want_feat=True, want_grad=True):
    """(d, z, grad d) of a given cell's MLP at x (no cell map)."""
    w = _f32(w)
    x = np.ascontiguousarray(x, dtype=np.float64)
    feat = np.zeros(g.feat_dim) if want_feat else None
    grad = np.zeros(3) if want_grad else None
    d = lib().ko_sdf_eval(C.byref(_desc(g)), _p(w, C.c_float), int(cell_id), _p(x, C.c_double),
                          _p(feat, C.c_double), _p(grad, C.c_double))
    return d, feat, grad


def sdf(g, w, pts):
    """Batch (d, z, grad d, cell) at points, cell chosen by m(x)."""
    w = _f32(w)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    n = pts.shape[0]
    d = np.zeros(n)
    feat = np.zeros((n, g.feat_dim))
    grad = np.zeros((n, 3))
    cells = np.zeros(n, dtype=np.int32)
    lib().ko_sdf_batch(C.byref(_desc(g)), _p(w, C.c_float), n, _p(pts, C.c_double), _p(d, C.c_double),
                       _p(feat, C.c_double), _p(grad, C.c_double), _p(cells, C.c_int32))
    return d, feat, grad, cells


def colour(g, w, cell_id, x, feat, n, v) -> np.ndarray:
    w = _f32(w)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, feat, n, v)]
    rgb = np.zeros(3)
    lib().ko_colour_eval(C.byref(_desc(g)), _p(w, C.c_float), int(cell_id), *[_p(a, C.c_double) for a in arrs],
                         _p(rgb, C.c_double))
    return rgb


def occupancy(g, w, res: int = None, thresh: float = None) -> np.ndarray:
    """Occupancy words (uint64, x-fastest bits): |d(voxel centre)| < voxel diagonal."""
    res = int(res or g.occ_res)
    if thresh is None:
        thresh = float(np.sqrt(sum(((g.bbox_max[a] - g.bbox_min[a]) / res) ** 2 for a in range(3))))
    nwords = (res ** 3 + 63) // 64
    bits = np.zeros(nwords, dtype=np.uint64)
    w = _f32(w)
    lib().ko_occupancy(C.byref(_desc(g)), _p(w, C.c_float), res, thresh, _p(bits, C.c_uint64))
    return bits


def ray(cam, i: int, j: int):
    cam = _f32(cam)
    o = np.zeros(3)
    d = np.zeros(3)
    lib().ko_ray(_p(cam, C.c_float), int(i), int(j), _p(o, C.c_double), _p(d, C.c_double))
    return o, d


def render(g, w, occ, cams, W: int, H: int, max_steps: int, eps: float, sel=None, delta_step: float = 0.0):
    """Sphere-trace the selected pixels (or all).  Returns a dict of per-ray arrays.

    occ: uint64 occupancy words or None (no empty-space skipping).
    sel: global pixel ids cam*H*W + i*W + j, or None for every pixel.
    delta_step: > 0 makes the margins conditioning-aware (see ko_trace_cond in kns_oracle.c):
    each margin then has the predicted deviation of a trajectory computed with per-step error
    delta_step subtracted.  0 gives the raw margins and skips the extra gradient evaluations.
    """
    w = _f32(w)
    cams = _f32(cams).reshape(-1, 16)
    occ = None if occ is None else np.ascontiguousarray(occ, dtype=np.uint64)
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        n = sel.size
    else:
        n = cams.shape[0] * W * H
    out = dict(rgb=np.zeros((n, 3), np.float32), depth=np.zeros(n, np.float32),
               normal=np.zeros((n, 3), np.float32), cell=np.zeros(n, np.int32), hit=np.zeros(n, np.uint8),
               steps=np.zeros(n, np.int32), margins=np.zeros((n, 4)), by_max=np.zeros(n, np.uint8))
    lib().ko_render(C.byref(_desc(g)), _p(w, C.c_float), _p(occ, C.c_uint64), _p(cams, C.c_float),
                    cams.shape[0], W, H, max_steps, eps, float(delta_step), n if sel is not None else 0,
                    _p(sel, C.c_int64),
                    _p(out["rgb"], C.c_float), _p(out["depth"], C.c_float), _p(out["normal"], C.c_float),
                    _p(out["cell"], C.c_int32), _p(out["hit"], C.c_uint8), _p(out["steps"], C.c_int32),
                    _p(out["margins"], C.c_double), _p(out["by_max"], C.c_uint8))
    return out


def trace_rays(g, w, occ, o, dirs, max_steps: int, eps: float):
    """Sphere-trace explicit rays (unit directions); FP64 outputs."""
    w = _f32(w)
    occ = None if occ is None else np.ascontiguousarray(occ, dtype=np.uint64)
    o = np.ascontiguousarray(o, dtype=np.float64).reshape(-1, 3)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    n = o.shape[0]
    out = dict(depth=np.zeros(n), cell=np.zeros(n, np.int32), steps=np.zeros(n, np.int32),
               normal=np.zeros((n, 3)), rgb=np.zeros((n, 3)))
    lib().ko_trace_rays(C.byref(_desc(g)), _p(w, C.c_float), _p(occ, C.c_uint64), n, _p(o, C.c_double),
                        _p(dirs, C.c_double), max_steps, eps, _p(out["depth"], C.c_double),
                        _p(out["cell"], C.c_int32), _p(out["steps"], C.c_int32), _p(out["normal"], C.c_double),
                        _p(out["rgb"], C.c_double))
    return out


def first_occupied(g, occ, o, w, t: float):
    """DDA from x(t) to the next occupied voxel: (t_entry, voxel ijk) or None."""
    occ = np.ascontiguousarray(occ, dtype=np.uint64)
    o = np.ascontiguousarray(o, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    te = np.zeros(1)
    v = np.zeros(3, dtype=np.int32)
    ok = lib().ko_first_occupied(C.byref(_desc(g)), _p(occ, C.c_uint64), _p(o, C.c_double), _p(w, C.c_double),
                                 float(t), _p(te, C.c_double), _p(v, C.c_int32))
    return (float(te[0]), tuple(int(a) for a in v)) if ok else None


def march_roots(g, w, o, dirs, t0, t1, dt: float = 1e-4, tol: float = 1e-12) -> np.ndarray:
    """Brute force: first sign change of d along each ray in [t0, t1], bisected to tol (NaN if none)."""
    w = _f32(w)
    o = np.ascontiguousarray(o, dtype=np.float64).reshape(-1, 3)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    n = o.shape[0]
    t0 = np.ascontiguousarray(np.broadcast_to(t0, (n,)), dtype=np.float64)
    t1 = np.ascontiguousarray(np.broadcast_to(t1, (n,)), dtype=np.float64)
    roots = np.zeros(n)
    lib().ko_march_roots(C.byref(_desc(g)), _p(w, C.c_float), n, _p(o, C.c_double), _p(dirs, C.c_double),
                         _p(t0, C.c_double), _p(t1, C.c_double), dt, tol, _p(roots, C.c_double))
    return roots


def robust_mask(margins: np.ndarray, delta_d: float, delta_x: float, delta_t: float = None) -> np.ndarray:
    """Rays whose every decision margin exceeds the given bounds (see kns_oracle.c header)."""
    delta_t = delta_x if delta_t is None else delta_t
    return ((margins[:, 0] > delta_d) & (margins[:, 1] > delta_t) & (margins[:, 2] > delta_x)
            & (margins[:, 3] > delta_x))


def train_loss(g, w, s: float, s_up: float, o, dirs, target, u_strat, u_imp, points, lam: float, h: float,
               t_fixed=None, want_t: bool = False, want_rgb: bool = False):
    """NeuS-style training loss (see ko_train_loss in kns_oracle.c).  Returns (loss, parts, t[, rgb])."""
    w = _f32(w)
    o = np.ascontiguousarray(o, dtype=np.float64).reshape(-1, 3)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    target = np.ascontiguousarray(target, dtype=np.float64).reshape(-1, 3)
    u_strat = np.ascontiguousarray(u_strat, dtype=np.float64)
    u_imp = np.ascontiguousarray(u_imp, dtype=np.float64)
    points = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    B, Ns, Ni = o.shape[0], u_strat.shape[1], u_imp.shape[1]
    tf = None if t_fixed is None else np.ascontiguousarray(t_fixed, dtype=np.float64)
    t_out = np.zeros((B, Ns + Ni)) if want_t else None
    rgb = np.zeros((B, 3)) if want_rgb else None
    parts = np.zeros(2)
    loss = lib().ko_train_loss(C.byref(_desc(g)), _p(w, C.c_float), float(s), float(s_up), B, _p(o, C.c_double),
                               _p(dirs, C.c_double), _p(target, C.c_double), Ns, _p(u_strat, C.c_double), Ni,
                               _p(u_imp, C.c_double), points.shape[0], _p(points, C.c_double), float(lam), float(h),
                               _p(tf, C.c_double), _p(t_out, C.c_double), _p(parts, C.c_double), _p(rgb, C.c_double))
    if want_rgb:
        return loss, parts, t_out, rgb
    return loss, parts, t_out


def train_grad(g, w, s: float, s_up: float, o, dirs, target, u_strat, u_imp, points, lam: float, h: float,
               t_fixed=None):
    """Loss and its reverse-mode gradient over every weight (see ko_train_grad).  Returns (loss, parts, grad)."""
    w = _f32(w)
    o = np.ascontiguousarray(o, dtype=np.float64).reshape(-1, 3)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    target = np.ascontiguousarray(target, dtype=np.float64).reshape(-1, 3)
    u_strat = np.ascontiguousarray(u_strat, dtype=np.float64)
    u_imp = np.ascontiguousarray(u_imp, dtype=np.float64)
    points = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    tf = None if t_fixed is None else np.ascontiguousarray(t_fixed, dtype=np.float64)
    grad = np.zeros(w.shape[0], dtype=np.float64)
    parts = np.zeros(2)
    loss = lib().ko_train_grad(C.byref(_desc(g)), _p(w, C.c_float), float(s), float(s_up), o.shape[0],
                               _p(o, C.c_double), _p(dirs, C.c_double), _p(target, C.c_double), u_strat.shape[1],
                               _p(u_strat, C.c_double), u_imp.shape[1], _p(u_imp, C.c_double), points.shape[0],
                               _p(points, C.c_double), float(lam), float(h), _p(tf, C.c_double), _p(grad, C.c_double),
                               _p(parts, C.c_double))
    return loss, parts, grad


def splitmix64(seed: int, k: int) -> int:
    return int(lib().ko_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, k))


def pt_uniform(seed: int, path: int, depth: int, dim: int) -> float:
    return float(lib().ko_pt_uniform(seed, path, depth, dim))


def cosine_dir(n, u1: float, u2: float) -> np.ndarray:
    n = np.ascontiguousarray(n, dtype=np.float64)
    w = np.zeros(3)
    lib().ko_cosine_dir(_p(n, C.c_double), float(u1), float(u2), _p(w, C.c_double))
    return w


def sky(w, horizon, zenith) -> np.ndarray:
    out = np.zeros(3)
    args = [np.ascontiguousarray(v, dtype=np.float64) for v in (w, horizon, zenith)]
    lib().ko_sky(*[_p(v, C.c_double) for v in args], _p(out, C.c_double))
    return out


def path_trace(g, w, occ, cams, W: int, H: int, spp: int, max_depth: int, max_steps: int, eps: float,
               offset: float, seed: int, horizon, zenith, sel=None):
    """Lambertian path tracing (see ko_path_trace).  Returns dict(rgb per pixel, L per path, traces per path)."""
    w = _f32(w)
    cams = _f32(cams).reshape(-1, 16)
    occ = None if occ is None else np.ascontiguousarray(occ, dtype=np.uint64)
    sel = np.arange(cams.shape[0] * W * H, dtype=np.int64) if sel is None else np.ascontiguousarray(sel, np.int64)
    n = sel.size
    hz = np.ascontiguousarray(horizon, dtype=np.float64)
    zn = np.ascontiguousarray(zenith, dtype=np.float64)
    out = dict(rgb=np.zeros((n, 3)), L=np.zeros((n, spp, 3)), traces=np.zeros((n, spp), np.int32))
    lib().ko_path_trace(C.byref(_desc(g)), _p(w, C.c_float), _p(occ, C.c_uint64), _p(cams, C.c_float),
                        cams.shape[0], W, H, spp, max_depth, max_steps, float(eps), float(offset), seed,
                        _p(hz, C.c_double), _p(zn, C.c_double), n, _p(sel, C.c_int64),
                        _p(out["rgb"], C.c_double), _p(out["L"], C.c_double), _p(out["traces"], C.c_int32))
    return out
