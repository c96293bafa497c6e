"""Seeded synthetic inputs for the KiloNeuS sphere-tracing path.

This module only draws numbers and lays them out; it holds none of the
method's arithmetic (no positional encoding, no MLP evaluation, no tracing).
Both the CUDA library and the FP64 oracle consume what it produces, so it must
not import either of them.

Random numbers come from a counter-based generator written out from its
published definition (SplitMix64, Steele, Lea & Flood, OOPSLA 2014): the
64-bit value for (key, i) is the SplitMix64 finaliser applied to
key + (i + 1) * 0x9E3779B97F4A7C15.  Keys are derived from (seed, stream) by
the same finaliser, so any language can reproduce every weight.  Normal
variates use the Box-Muller cosine branch on a pair of uniforms.

Weight layout ("canonical", FP32, the layout every API takes): cells in
x-fastest order (cell = ix + N*(iy + N*iz)); per cell, the SDF MLP layers then
the colour MLP layers; per layer, W[out][in] row-major followed by b[out].

The SDF weights follow the geometric (SAL) initialisation for a sphere of
radius 0.5 with one base draw shared by every cell plus a per-cell N(0, std)
perturbation, so the global zero level set is a near-sphere whose cells differ
slightly (the Kilo-grid of Sec. 3.1 with independent per-cell MLPs).  Colour
weights are drawn independently per cell, so a wrong cell index is visible in
the rendered colour.
"""
from __future__ import annotations

import dataclasses
import math
import struct
from typing import List, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1

# generator streams (documented so other implementations can reproduce them)
STREAM_SDF_BASE = 1
STREAM_SDF_CELL = 2
STREAM_COL_CELL = 3
STREAM_CAMERA = 4
STREAM_POINTS = 5
STREAM_TRAIN = 7


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _mix_int(x: int) -> int:
    z = x & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int, sub: int = 0) -> int:
    """64-bit key of generator stream (seed, stream, sub)."""
    k = _mix_int((seed * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) & _MASK)
    k = _mix_int((k ^ (stream * 0xD1B54A32D192ED03)) & _MASK)
    return _mix_int((k ^ ((sub + 1) * 0x8CB92BA72F3D8DD7)) & _MASK)


def u64(key: int, start: int, count: int) -> np.ndarray:
    i = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (i + np.uint64(1)) * _GAMMA
    return _mix(z)


def uniform(key: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (u64(key, start, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(key: int, count: int, start: int = 0) -> np.ndarray:
    """Standard normals: Box-Muller (cos branch) on uniforms 2i and 2i+1."""
    u = u64(key, 2 * start, 2 * count)
    u1 = ((u[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53  # (0, 1]
    u2 = (u[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _u64_rows(keys: np.ndarray, count: int) -> np.ndarray:
    i = np.arange(count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = keys[:, None] + (i[None, :] + np.uint64(1)) * _GAMMA
    return _mix(z)


def _uniform_rows(keys: np.ndarray, count: int) -> np.ndarray:
    """uniform(key, count) for each key in keys, stacked as rows."""
    return (_u64_rows(keys, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def _normal_rows(keys: np.ndarray, count: int) -> np.ndarray:
    """normal(key, count) for each key in keys, stacked as rows."""
    u = _u64_rows(keys, 2 * count)
    u1 = ((u[:, 0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (u[:, 1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclasses.dataclass(frozen=True)
class GridDesc:
    """Shape of a Kilo-grid (Sec. 3.1): N^3 cells, each with an SDF MLP and a colour MLP."""
    N: int = 8
    pe_pos_L: int = 4
    pe_dir_L: int = 2
    sdf_hidden: int = 2
    sdf_width: int = 32
    feat_dim: int = 15
    col_hidden: int = 1
    col_width: int = 32
    col_use_x: int = 0
    occ_res: int = 0
    softplus_beta: float = 100.0
    bbox_min: Tuple[float, float, float] = (-1.0, -1.0, -1.0)
    bbox_max: Tuple[float, float, float] = (1.0, 1.0, 1.0)

    @property
    def n_cells(self) -> int:
        return self.N ** 3

    @property
    def sdf_in(self) -> int:
        return 3 + 6 * self.pe_pos_L

    @property
    def col_in(self) -> int:
        return self.feat_dim + 3 + (3 + 6 * self.pe_dir_L) + (3 if self.col_use_x else 0)

    def sdf_layers(self) -> List[Tuple[int, int]]:
        """(in, out) of each SDF layer; the last one outputs [d, z_0..z_{feat_dim-1}]."""
        dims = [self.sdf_in] + [self.sdf_width] * self.sdf_hidden + [1 + self.feat_dim]
        return list(zip(dims[:-1], dims[1:]))

    def col_layers(self) -> List[Tuple[int, int]]:
        dims = [self.col_in] + [self.col_width] * self.col_hidden + [3]
        return list(zip(dims[:-1], dims[1:]))

    @property
    def p_sdf(self) -> int:
        return sum(i * o + o for i, o in self.sdf_layers())

    @property
    def p_col(self) -> int:
        return sum(i * o + o for i, o in self.col_layers())

    @property
    def p_cell(self) -> int:
        return self.p_sdf + self.p_col


def layer_offsets(desc: GridDesc):
    """Offsets (within one cell's block) of (W, b) for each SDF and colour layer."""
    out = []
    off = 0
    for i, o in desc.sdf_layers() + desc.col_layers():
        out.append((off, off + i * o, i, o))
        off += i * o + o
    return out


def sal_sphere_grid(desc: GridDesc, seed: int = 0, perturb_std: float = 1e-3,
                    radius: float = 0.5) -> np.ndarray:
    """Canonical FP32 weights: SAL sphere init (radius r) + per-cell N(0, perturb_std).

    SAL-style initialisation: hidden W ~ N(0, sqrt(2)/sqrt(out)), b = 0; the first
    layer's sin/cos columns are zero so only the raw xyz columns are drawn; the
    last layer's d row ~ N(sqrt(pi)/sqrt(in), 1e-4) with bias -r; the feature rows
    ~ N(0, 1/sqrt(in)) with bias 0.  The colour MLP is drawn per cell from
    U(-1/sqrt(in), 1/sqrt(in)) for weights and biases.
    """
    nc = desc.n_cells
    base = np.zeros(desc.p_sdf, dtype=np.float64)
    key = stream_key(seed, STREAM_SDF_BASE)
    off = 0
    cursor = 0
    layers = desc.sdf_layers()
    for li, (i, o) in enumerate(layers):
        n = i * o
        z = normal(key, n + o, start=cursor)
        cursor += n + o
        Wl = z[:n].reshape(o, i)
        if li == len(layers) - 1:
            Wl = Wl.copy()
            Wl[0, :] = math.sqrt(math.pi) / math.sqrt(i) + 1e-4 * Wl[0, :]
            Wl[1:, :] = Wl[1:, :] / math.sqrt(i)
            bl = np.zeros(o)
            bl[0] = -radius
        else:
            Wl = Wl * (math.sqrt(2.0) / math.sqrt(o))
            if li == 0:
                Wl = Wl.copy()
                Wl[:, 3:] = 0.0
            bl = np.zeros(o)
        base[off:off + n] = Wl.reshape(-1)
        base[off + n:off + n + o] = bl
        off += n + o
    assert off == desc.p_sdf

    w = np.empty((nc, desc.p_cell), dtype=np.float32)
    col_scale = np.concatenate([np.full(i * o + o, 1.0 / math.sqrt(i)) for i, o in desc.col_layers()])
    chunk = 1024
    for c0 in range(0, nc, chunk):
        cells = range(c0, min(nc, c0 + chunk))
        pk = np.array([stream_key(seed, STREAM_SDF_CELL, c) for c in cells], dtype=np.uint64)
        ck = np.array([stream_key(seed, STREAM_COL_CELL, c) for c in cells], dtype=np.uint64)
        w[c0:c0 + len(pk), :desc.p_sdf] = (base[None, :] + perturb_std * _normal_rows(pk, desc.p_sdf)
                                           ).astype(np.float32)
        u = _uniform_rows(ck, desc.p_col)
        w[c0:c0 + len(pk), desc.p_sdf:] = ((2.0 * u - 1.0) * col_scale[None, :]).astype(np.float32)
    return w.reshape(-1)


# ---------------------------------------------------------------- cameras
CAMERA_FLOATS = 16  # c2w[12] row-major 3x4, fx, fy, cx, cy


def look_at_camera(pos, W: int, H: int, vfov_deg: float = 40.0, target=(0.0, 0.0, 0.0),
                   up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Pinhole camera as 16 floats: c2w (3x4, columns = right, down, forward, position), fx, fy, cx, cy.

    Camera frame: x right, y down, z forward; pixel (i, j) = (row, column) with row 0 at the top.
    """
    pos = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=1)
    c2w = np.concatenate([R, pos[:, None]], axis=1)
    fy = (H / 2.0) / math.tan(math.radians(vfov_deg) / 2.0)
    cam = np.concatenate([c2w.reshape(-1), [fy, fy, W / 2.0, H / 2.0]])
    return cam.astype(np.float32)


def orbit_cameras(n: int, W: int, H: int, seed: int = 1, radius: float = 2.5,
                  evenly_spaced: bool = False, vfov_deg: float = 40.0) -> np.ndarray:
    """n seeded orbit cameras looking at the origin, elevation U(-30, 30) degrees.

    evenly_spaced: azimuth 2*pi*k/n + U(-10, 10) degrees; otherwise azimuth U(0, 2*pi).
    """
    u = uniform(stream_key(seed, STREAM_CAMERA), 2 * n)
    cams = []
    for k in range(n):
        if evenly_spaced:
            az = 2.0 * math.pi * k / n + math.radians(20.0 * u[2 * k] - 10.0)
        else:
            az = 2.0 * math.pi * u[2 * k]
        el = math.radians(60.0 * u[2 * k + 1] - 30.0)
        pos = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az),
                                 math.sin(el)])
        cams.append(look_at_camera(pos, W, H, vfov_deg))
    return np.stack(cams).astype(np.float32)


def uniform_points(n: int, seed: int, lo=-1.0, hi=1.0) -> np.ndarray:
    """n points uniform in the box [lo, hi]^3 (FP32, n x 3)."""
    u = uniform(stream_key(seed, STREAM_POINTS), 3 * n).reshape(n, 3)
    return (lo + (hi - lo) * u).astype(np.float32)


# ---------------------------------------------------------------- workloads
def config_desc(name: str) -> GridDesc:
    """Grid shapes of the named synthetic workloads."""
    if name == "c1":   # 8^3 grid, 2 hidden layers of width 32, no occupancy
        return GridDesc(N=8, sdf_hidden=2, sdf_width=32, col_width=32, occ_res=0)
    if name == "c2":   # 16^3 grid, 3 hidden layers of width 32, 128^3 occupancy
        return GridDesc(N=16, sdf_hidden=3, sdf_width=32, col_width=32, occ_res=128)
    if name == "c3s":  # 16^3 grid, width 32 (the BF16 small form)
        return GridDesc(N=16, sdf_hidden=3, sdf_width=32, col_width=32, occ_res=128)
    if name == "c3l":  # 32^3 grid, width 64 (the BF16 large form)
        return GridDesc(N=32, sdf_hidden=3, sdf_width=64, col_width=64, occ_res=128)
    raise KeyError(name)


WORKLOADS = {
    # name: (grid, n_cams, W, H, max_steps, eps, evenly_spaced cameras)
    "c1": ("c1", 4, 64, 64, 64, 1e-4, True),
    "c2": ("c2", 8, 800, 800, 128, 1e-4, False),
    "c3s": ("c3s", 8, 1920, 1080, 128, 1e-4, False),
    "c3l": ("c3l", 8, 1920, 1080, 128, 1e-4, False),
}


def workload(name: str, seed: int = 0):
    """(desc, weights, cameras, W, H, max_steps, eps) of a named workload."""
    gname, n_cams, W, H, max_steps, eps, even = WORKLOADS[name]
    desc = config_desc(gname)
    w = sal_sphere_grid(desc, seed=seed)
    cams = orbit_cameras(n_cams, W, H, seed=seed + 1, evenly_spaced=even)
    return desc, w, cams, W, H, max_steps, eps


# ---------------------------------------------------------------- .kns file
KNS_MAGIC = b"KNS1"
KNS_VERSION = 1


def write_kns(path: str, desc: GridDesc, weights: np.ndarray, occ_bits: np.ndarray = None) -> None:
    """Write a versioned grid file: header, canonical FP32 weights, optional occupancy words.

    Header (little-endian): magic "KNS1", u32 version, 10 x i32 (N, pe_pos_L, pe_dir_L,
    sdf_hidden, sdf_width, feat_dim, col_hidden, col_width, col_use_x, occ_res),
    7 x f32 (softplus_beta, bbox_min[3], bbox_max[3]), u64 n_floats, u64 n_occ_words.
    """
    weights = np.ascontiguousarray(weights, dtype=np.float32)
    occ = None if occ_bits is None else np.ascontiguousarray(occ_bits, dtype=np.uint64)
    with open(path, "wb") as f:
        f.write(KNS_MAGIC)
        f.write(struct.pack("<I", KNS_VERSION))
        f.write(struct.pack("<10i", desc.N, desc.pe_pos_L, desc.pe_dir_L, desc.sdf_hidden,
                            desc.sdf_width, desc.feat_dim, desc.col_hidden, desc.col_width,
                            desc.col_use_x, desc.occ_res))
        f.write(struct.pack("<7f", desc.softplus_beta, *desc.bbox_min, *desc.bbox_max))
        f.write(struct.pack("<QQ", weights.size, 0 if occ is None else occ.size))
        f.write(weights.tobytes())
        if occ is not None:
            f.write(occ.tobytes())


# ---------------------------------------------------------------- training batches
# The fine-tuning workload: 2^18 rays through a 16^3 grid of width-32 MLPs (3 hidden layers), 64
# stratified + 32 importance samples per ray, L1 colour + 0.1 x eikonal on 2^16 uniform points.  The
# rays are random pixels of 8 orbit cameras at 800 x 800; the targets are renders of a perturbed
# sphere grid (seed 3, per-cell perturbation std 1e-2); the trained weights start from the SAL grid.
TRAIN_WORKLOAD = dict(grid="c2", n_rays=1 << 18, n_strat=64, n_imp=32, n_eik=1 << 16, s=20.0, s_up=64.0,
                      lam=0.1, h=1e-2, n_cams=8, W=800, H=800, max_steps=128, eps=1e-4, target_seed=3,
                      target_std=1e-2)


def pixel_rays(cams: np.ndarray, W: int, H: int, sel: np.ndarray):
    """Origins and unit directions (FP32, n x 3) of global pixel ids cam*H*W + i*W + j (pixel centres)."""
    cams = np.asarray(cams, dtype=np.float64).reshape(-1, 16)
    sel = np.asarray(sel, dtype=np.int64)
    c = sel // (W * H)
    i = (sel // W) % H
    j = sel % W
    cam = cams[c]
    dx = (j + 0.5 - cam[:, 14]) / cam[:, 12]
    dy = (i + 0.5 - cam[:, 15]) / cam[:, 13]
    R = cam[:, :12].reshape(-1, 3, 4)
    d = R[:, :, 0] * dx[:, None] + R[:, :, 1] * dy[:, None] + R[:, :, 2]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return R[:, :, 3].astype(np.float32), d.astype(np.float32)


def train_draws(n_rays: int, n_strat: int, n_imp: int, n_eik: int, n_pix: int, seed: int):
    """Seeded random draws of one training batch (FP32): pixel ids, stratified jitter (n_rays x n_strat),
    ascending importance uniforms (n_rays x n_imp) and eikonal points uniform in [-1, 1]^3."""
    sel = (uniform(stream_key(seed, STREAM_TRAIN, 0), n_rays) * n_pix).astype(np.int64)
    u_s = uniform(stream_key(seed, STREAM_TRAIN, 1), n_rays * n_strat).reshape(n_rays, n_strat)
    u_i = np.sort(uniform(stream_key(seed, STREAM_TRAIN, 2), n_rays * n_imp).reshape(n_rays, n_imp), axis=1)
    pts = uniform(stream_key(seed, STREAM_TRAIN, 3), 3 * n_eik).reshape(n_eik, 3) * 2.0 - 1.0
    # FP32 rounding can tie neighbours but keeps the rows ascending
    return sel, u_s.astype(np.float32), u_i.astype(np.float32), pts.astype(np.float32)
