"""Hand-built Kilo-grid weights whose fields have closed forms (test inputs only).

The patterns rely on two exact identities of the activations (Sec. 3.1):
  softplus_b(s) - softplus_b(-s) = s   and   relu(s) - relu(-s) = s.
Routing a value through a hidden layer as a (+s, -s) unit pair therefore
carries it through every layer unchanged, so the whole SDF MLP collapses to a
linear function of x (an exact plane), and the colour MLP to a sigmoid of a
linear function of chosen inputs.  Pair units are placed at scattered,
asymmetric positions so that a transposed weight read or an off-by-one index
breaks the identity.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2206_10885_gb300 import synth as S


def pair_units(layer: int, width: int):
    """Output units carrying (+s, -s) after hidden layer `layer` (scattered, asymmetric)."""
    p0 = (7 * layer + 1) % width
    p1 = (7 * layer + 4 + (layer % 3)) % width
    if p1 == p0:
        p1 = (p0 + 1) % width
    return p0, p1


def plane_grid(desc: S.GridDesc, a, b, feat_c=None, feat_e=None, cell_b=None) -> np.ndarray:
    """SDF of every cell = a.x + b (or a.x + cell_b[cell]); features z_j = c_j (a.x + b) + e_j.

    The colour MLP is zero (RGB = sigmoid(0) = 0.5) unless overwritten.
    """
    a = np.asarray(a, dtype=np.float64)
    nc = desc.n_cells
    w = np.zeros((nc, desc.p_cell), dtype=np.float64)
    offs = S.layer_offsets(desc)
    ns = len(desc.sdf_layers())
    feat_c = np.zeros(desc.feat_dim) if feat_c is None else np.asarray(feat_c, dtype=np.float64)
    feat_e = np.zeros(desc.feat_dim) if feat_e is None else np.asarray(feat_e, dtype=np.float64)
    width = desc.sdf_width
    for li in range(ns):
        wo, bo, nin, nout = offs[li]
        Wl = np.zeros((nout, nin))
        bl = np.zeros((nc, nout))
        if li == 0:
            q0, q1 = pair_units(0, width)
            Wl[q0, 0:3] = a
            Wl[q1, 0:3] = -a
            bb = np.full(nc, float(b)) if cell_b is None else np.asarray(cell_b, dtype=np.float64)
            bl[:, q0] = bb
            bl[:, q1] = -bb
        elif li < ns - 1:
            p0, p1 = pair_units(li - 1, width)
            q0, q1 = pair_units(li, width)
            Wl[q0, p0], Wl[q0, p1] = 1.0, -1.0
            Wl[q1, p0], Wl[q1, p1] = -1.0, 1.0
        else:
            p0, p1 = pair_units(li - 1, width)
            Wl[0, p0], Wl[0, p1] = 1.0, -1.0
            for j in range(desc.feat_dim):
                Wl[1 + j, p0], Wl[1 + j, p1] = feat_c[j], -feat_c[j]
                bl[:, 1 + j] = feat_e[j]
        w[:, wo:bo] = Wl.reshape(-1)[None, :]
        w[:, bo:bo + nout] = bl
    return w.astype(np.float32).reshape(-1)


def set_colour_linear(desc: S.GridDesc, w: np.ndarray, inputs, K, bias, cell_bias=None) -> np.ndarray:
    """Colour MLP: logits = K @ u[inputs] + bias (+ cell_bias[cell]) via relu pairs.

    inputs: indices into the colour input u = [z, n, gamma(v), x?]; K: 3 x len(inputs).
    Requires one hidden layer of width >= 2*len(inputs).
    """
    assert desc.col_hidden == 1 and desc.col_width >= 2 * len(inputs)
    w = w.reshape(desc.n_cells, desc.p_cell).copy()
    offs = S.layer_offsets(desc)
    ns = len(desc.sdf_layers())
    (w0, b0, i0, o0), (w1, b1, i1, o1) = offs[ns], offs[ns + 1]
    W0 = np.zeros((o0, i0))
    W1 = np.zeros((o1, i1))
    for m, src in enumerate(inputs):
        u0, u1 = (5 * (2 * m) + 3) % o0, (5 * (2 * m + 1) + 3) % o0  # a scrambled permutation
        W0[u0, src], W0[u1, src] = 1.0, -1.0
        for r in range(3):
            W1[r, u0], W1[r, u1] = K[r][m], -K[r][m]
    w[:, w0:b0] = W0.reshape(-1)[None, :]
    w[:, b0:b0 + o0] = 0.0
    w[:, w1:b1] = W1.reshape(-1)[None, :]
    bb = np.tile(np.asarray(bias, dtype=np.float64), (desc.n_cells, 1))
    if cell_bias is not None:
        bb = bb + np.asarray(cell_bias, dtype=np.float64)
    w[:, b1:b1 + 3] = bb
    return w.astype(np.float32).reshape(-1)


def pe_pick_grid(desc: S.GridDesc, column: int, scale: float = 1.0, offset: float = 0.0) -> np.ndarray:
    """SDF = scale * gamma(x)[column] + offset in every cell (picks one encoding column)."""
    w = plane_grid(desc, [0.0, 0.0, 0.0], 0.0).reshape(desc.n_cells, desc.p_cell)
    wo, bo, nin, nout = S.layer_offsets(desc)[0]
    q0, q1 = pair_units(0, desc.sdf_width)
    W0 = np.zeros((nout, nin))
    W0[q0, column] = scale
    W0[q1, column] = -scale
    w[:, wo:bo] = W0.reshape(-1)[None, :]
    b0 = np.zeros(nout)
    b0[q0], b0[q1] = offset, -offset
    w[:, bo:bo + nout] = b0[None, :]
    return w.astype(np.float32).reshape(-1)


def random_grid(desc: S.GridDesc, seed: int, scale: float = 0.5) -> np.ndarray:
    """Dense random weights in every layer (every PE column and unit live)."""
    u = S.uniform(S.stream_key(seed, 99), desc.n_cells * desc.p_cell)
    return ((2.0 * u - 1.0) * scale).astype(np.float32)


def sigmoid(s):
    return 1.0 / (1.0 + np.exp(-np.asarray(s, dtype=np.float64)))


def fib_dirs(n: int) -> np.ndarray:
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = math.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def plane_side_cameras(a, n: int, W: int, H: int, seed: int) -> np.ndarray:
    """Cameras at radius 2.5 on the positive side of the plane a.x + b (looking at the origin)."""
    rng = np.random.default_rng(seed)
    a = np.asarray(a, dtype=np.float64)
    cams = []
    for _ in range(n):
        p = a + 0.35 * rng.normal(size=3)
        p = 2.5 * p / np.linalg.norm(p)
        cams.append(S.look_at_camera(p, W, H))
    return np.stack(cams)
