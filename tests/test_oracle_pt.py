"""Pins of the oracle's Lambertian path tracer (CPU only).

  * SplitMix64 against its published outputs for seed 0;
  * cosine-weighted directions: unit length, in the normal's hemisphere, E[cos] = 2/3, E[w] = 2n/3;
  * the sky gradient at the zenith, the nadir and the horizon;
  * a plane under a constant sky: a path that misses returns the sky E, one that hits and bounces
    returns albedo * E (the bounce leaves the plane and escapes), a hit at the last depth returns 0;
  * a plane under the sky gradient: the mean over many paths is albedo * (horizon / 6 + 5 zenith / 6).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2206_10885_gb300 import synth as S
from tests import gridkit as K


def test_splitmix64_published_outputs():
    assert [oracle.splitmix64(0, k) for k in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                          0x06C45D188009454F]


def test_uniforms_are_24_bit_fractions():
    u = np.array([oracle.pt_uniform(7, p, d, i) for p in range(50) for d in range(3) for i in range(4)])
    assert np.all((u >= 0) & (u < 1))
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))
    assert 0.4 < u.mean() < 0.6


@pytest.mark.parametrize("n", [(0, 0, 1), (0, 0, -1), (0.6, 0, 0.8), (-0.48, 0.6, -0.64), (1, 0, 0)])
def test_cosine_directions(n):
    n = np.asarray(n, dtype=np.float64)
    n /= np.linalg.norm(n)
    m = 64
    g = (np.arange(m) + 0.5) / m
    ws = np.array([oracle.cosine_dir(n, u1, u2) for u1 in g for u2 in g])
    np.testing.assert_allclose(np.linalg.norm(ws, axis=1), 1.0, atol=1e-12)
    cos = ws @ n
    assert cos.min() >= 0.0
    assert cos.mean() == pytest.approx(2.0 / 3.0, abs=2e-4)
    np.testing.assert_allclose(ws.mean(0), 2.0 / 3.0 * n, atol=2e-4)


def test_sky_gradient():
    h, z = np.array([1.0, 0.9, 0.8]), np.array([0.2, 0.4, 1.0])
    np.testing.assert_allclose(oracle.sky([0, 0, 1], h, z), z)
    np.testing.assert_allclose(oracle.sky([0, 0, -1], h, z), h)
    np.testing.assert_allclose(oracle.sky([1, 0, 0], h, z), 0.5 * (h + z))


def plane_scene(logit):
    desc = S.GridDesc(N=2, sdf_hidden=2, sdf_width=32, col_hidden=1, col_width=32, occ_res=0)
    w = K.plane_grid(desc, [0.0, 0.0, 1.0], -0.1)          # d = z - 0.1, normal +z
    w = K.set_colour_linear(desc, w, [0], [[0.0], [0.0], [0.0]], logit)
    cams = np.stack([S.look_at_camera([0.3, 0.2, 2.5], 12, 10), S.look_at_camera([-1.5, 1.2, 1.4], 12, 10)])
    return desc, w, cams


@pytest.mark.parametrize("max_depth", [1, 2, 3])
def test_plane_under_constant_sky(max_depth):
    logit = [0.4, -0.2, 1.3]
    desc, w, cams = plane_scene(logit)
    E = np.array([0.7, 0.8, 0.9])
    out = oracle.path_trace(desc, w, None, cams, 12, 10, 3, max_depth, 128, 1e-4, 1e-2, 5, E, E)
    albedo = K.sigmoid(np.float32(logit))
    L, tr = out["L"], out["traces"]
    miss = tr == 1
    hit_first = ~miss | (np.abs(L).sum(-1) == 0)
    assert miss.any() and (tr >= 1).all()
    if max_depth == 1:
        # one trace: sky on a miss, nothing on a hit
        for v in L.reshape(-1, 3):
            assert np.allclose(v, E, atol=1e-15) or np.all(v == 0)
        assert (np.abs(L).sum(-1) == 0).any()
    else:
        # a hit bounces once and escapes: albedo * E; never more than two traces
        assert tr.max() == 2
        np.testing.assert_allclose(L[tr == 1], np.broadcast_to(E, L[tr == 1].shape), atol=1e-15)
        np.testing.assert_allclose(L[tr == 2], np.broadcast_to(albedo * E, L[tr == 2].shape), rtol=1e-12)
    assert hit_first.any()
    np.testing.assert_allclose(out["rgb"], L.mean(1), atol=1e-15)


def test_plane_under_sky_gradient_mean():
    logit = [0.4, -0.2, 1.3]
    desc, w, cams = plane_scene(logit)
    cams = cams[:1]
    h, z = np.array([1.0, 0.9, 0.8]), np.array([0.2, 0.4, 1.0])
    sel = np.array([5 * 12 + 6])  # a pixel whose rays all hit the plane
    out = oracle.path_trace(desc, w, None, cams, 12, 10, 20000, 2, 128, 1e-4, 1e-2, 11, h, z, sel=sel)
    assert (out["traces"] == 2).all()
    albedo = K.sigmoid(np.float32(logit))
    np.testing.assert_allclose(out["rgb"][0], albedo * (h / 6 + 5 * z / 6), atol=4e-3)
