"""The seeded input generator (CPU only), pinned to its published definition and to the camera
conventions the renders assume."""
from __future__ import annotations

import math

import numpy as np

from paper_2206_10885_gb300 import synth as S


def test_splitmix64_published_outputs():
    # the generator with key 0 is SplitMix64 seeded with 0 (Steele, Lea & Flood 2014)
    assert [int(v) for v in S.u64(0, 0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # counter-based: any window of the sequence is the same values
    assert np.array_equal(S.u64(12345, 7, 5), S.u64(12345, 0, 12)[7:])


def test_scalar_and_vector_finalisers_agree():
    keys = [0, 1, 2 ** 63, 0xDEADBEEFCAFEF00D, S.stream_key(3, 4, 5)]
    assert [S._mix_int(k) for k in keys] == [int(v) for v in S._mix(np.array(keys, dtype=np.uint64))]


def test_row_generators_equal_the_single_key_ones():
    keys = np.array([S.stream_key(1, 2, c) for c in range(5)], dtype=np.uint64)
    u = S._uniform_rows(keys, 9)
    n = S._normal_rows(keys, 7)
    for r, k in enumerate(keys):
        assert np.array_equal(u[r], S.uniform(int(k), 9))
        assert np.array_equal(n[r], S.normal(int(k), 7))


def test_uniform_and_normal_distributions():
    u = S.uniform(S.stream_key(0, 1), 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))           # 53-bit fractions
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(u))
    z = S.normal(S.stream_key(0, 2), 200000)
    assert abs(z.mean()) < 4 / math.sqrt(len(z))
    assert abs(z.std() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.1                           # Gaussian kurtosis
    # streams and seeds are independent draws
    assert not np.array_equal(S.uniform(S.stream_key(0, 1), 8), S.uniform(S.stream_key(0, 2), 8))
    assert not np.array_equal(S.uniform(S.stream_key(0, 1), 8), S.uniform(S.stream_key(1, 1), 8))


def test_canonical_layout_sizes():
    for name in ("c1", "c2", "c3l"):
        desc = S.config_desc(name)
        offs = S.layer_offsets(desc)
        per_cell = offs[-1][1] + offs[-1][3]
        # SDF: (3 + 6 L) -> W ... -> 1 + 15; colour: [z, n, gamma_2(v)] = 33 -> W -> 3
        sdf = (27 * desc.sdf_width + desc.sdf_width + (desc.sdf_hidden - 1) * (desc.sdf_width + 1) * desc.sdf_width
               + (desc.sdf_width + 1) * 16)
        col = 33 * desc.col_width + desc.col_width + (desc.col_width + 1) * 3
        assert per_cell == sdf + col
        if name == "c1":  # (the larger grids take long to draw; their layout is the same code)
            w = S.sal_sphere_grid(desc)
            assert w.dtype == np.float32 and w.size == desc.N ** 3 * per_cell
    # c2: 4,723 parameters per cell
    assert S.layer_offsets(S.config_desc("c2"))[-1][1] + 3 == 4723


def test_orbit_cameras_follow_the_stated_convention():
    W, H = 800, 600
    cams = S.orbit_cameras(8, W, H, seed=1)
    assert cams.shape == (8, 16) and cams.dtype == np.float32
    for cam in cams.astype(np.float64):
        c2w = cam[:12].reshape(3, 4)
        right, down, fwd, pos = c2w[:, 0], c2w[:, 1], c2w[:, 2], c2w[:, 3]
        assert abs(np.linalg.norm(pos) - 2.5) < 1e-5                      # orbit radius
        np.testing.assert_allclose(fwd, -pos / np.linalg.norm(pos), atol=1e-6)  # looks at the origin
        np.testing.assert_allclose(c2w[:, :3].T @ c2w[:, :3], np.eye(3), atol=1e-6)
        assert abs(right[2]) < 1e-6                                       # world up +z: right is level
        assert down[2] <= 1e-6                                            # image rows go down
        elev = math.degrees(math.asin(pos[2] / 2.5))
        assert -30.0 - 1e-3 <= elev <= 30.0 + 1e-3
        fy = (H / 2) / math.tan(math.radians(20.0))                        # vertical FOV 40 degrees
        np.testing.assert_allclose(cam[12:], [fy, fy, W / 2, H / 2], rtol=1e-6)
    assert np.array_equal(cams, S.orbit_cameras(8, W, H, seed=1))
    assert not np.array_equal(cams, S.orbit_cameras(8, W, H, seed=2))


def test_pixel_rays_through_pixel_centres():
    W, H = 64, 48
    cams = S.orbit_cameras(2, W, H, seed=3)
    sel = np.array([0, W - 1, (H // 2) * W + W // 2, W * H + 5 * W + 7])
    o, d = S.pixel_rays(cams, W, H, sel)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    np.testing.assert_allclose(o[0], cams[0, [3, 7, 11]])
    np.testing.assert_allclose(o[3], cams[1, [3, 7, 11]])
    # the principal point is the image centre: the centre pixel's ray is the forward axis, offset by
    # half a pixel (pixel centres at j + 1/2, i + 1/2)
    c = cams[0].astype(np.float64)
    R = c[:12].reshape(3, 4)[:, :3]
    local = R.T @ d[2].astype(np.float64)
    local /= local[2]
    np.testing.assert_allclose(local[:2], [0.5 / c[12], 0.5 / c[13]], atol=1e-6)
    # the top-left pixel looks up and left, the top-right one up and right
    l0 = R.T @ d[0].astype(np.float64)
    l1 = R.T @ d[1].astype(np.float64)
    assert l0[0] < 0 and l0[1] < 0 and l1[0] > 0 and l1[1] < 0
