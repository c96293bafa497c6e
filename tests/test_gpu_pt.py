"""Explicit-ray tracing (kns_trace_rays) and Lambertian path tracing (kns_path_trace) against the FP64
oracle: closed forms on a plane, per-ray trace parity, per-pixel path-traced images."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2206_10885_gb300 import synth as S
from tests import gridkit as K

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_10885_gb300 as kns
    return kns


@pytest.fixture(scope="module")
def ctx(kns):
    c = kns.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_trace_rays_matches_oracle(kns, ctx):
    desc = S.config_desc("c2")
    w = S.sal_sphere_grid(desc, seed=0)
    grid = kns.Grid.load(ctx, desc, w)
    try:
        occ = grid.occupancy()
        rng = np.random.default_rng(3)
        # camera rays from outside, and rays starting inside the box in every direction
        cams = S.orbit_cameras(2, 32, 24, seed=5)
        o1, d1 = S.pixel_rays(cams, 32, 24, rng.integers(0, 2 * 32 * 24, 1500))
        o2 = rng.uniform(-0.9, 0.9, (1500, 3)).astype(np.float32)
        d2 = rng.normal(size=(1500, 3))
        d2 = (d2 / np.linalg.norm(d2, axis=1, keepdims=True)).astype(np.float32)
        o, d = np.concatenate([o1, o2]), np.concatenate([d1, d2])
        out = kns.trace_rays(ctx, grid, dev(o), dev(d), 128, 1e-4)
        torch.cuda.synchronize()
        ref = oracle.trace_rays(desc, w, occ, o.astype(np.float64), d.astype(np.float64), 128, 1e-4)
        hit = out["hit"].cpu().numpy().astype(bool)
        ref_hit = ref["cell"] >= 0
        assert np.mean(hit == ref_hit) >= 0.995
        both = hit & ref_hit
        assert both.sum() > 200 and (~ref_hit).sum() > 200
        depth = out["depth"].cpu().numpy()
        assert np.mean(np.abs(depth[both] - ref["depth"][both]) <= 1e-4) >= 0.99
        assert np.mean(np.abs(out["rgb"].cpu().numpy()[both] - ref["rgb"][both]).max(1) <= 1e-4) >= 0.99
        assert np.all(np.isinf(depth[~hit]))
        # the same rays through kns_render's camera path give the same hits
        img = kns.render(ctx, grid, cams, 32, 24, 128, 1e-4)
        sel = rng.integers(0, 2 * 32 * 24, 200)
        ot, dt = S.pixel_rays(cams, 32, 24, sel)
        tr = kns.trace_rays(ctx, grid, dev(ot), dev(dt), 128, 1e-4)
        assert np.mean(tr["hit"].cpu().numpy() == img["hit"].cpu().numpy()[sel]) >= 0.99
        # empty and bad calls
        kns.capi.kns_trace_rays(ctx.handle, grid.handle, 0, 0, 0, 128, 1e-4, kns.alloc_frame(1)[1])
        with pytest.raises(kns.KnsError):
            kns.capi.kns_trace_rays(ctx.handle, grid.handle, 0, 0, 5, 128, 1e-4, kns.alloc_frame(5)[1])
    finally:
        grid.free()


def plane_scene(logit):
    desc = S.GridDesc(N=2, sdf_hidden=2, sdf_width=32, col_hidden=1, col_width=32, occ_res=0)
    w = K.plane_grid(desc, [0.0, 0.0, 1.0], -0.1)
    w = K.set_colour_linear(desc, w, [0], [[0.0], [0.0], [0.0]], logit)
    cams = np.stack([S.look_at_camera([0.3, 0.2, 2.5], 12, 10), S.look_at_camera([-1.5, 1.2, 1.4], 12, 10)])
    return desc, w, cams


def test_path_trace_plane_closed_forms(kns, ctx):
    logit = [0.4, -0.2, 1.3]
    desc, w, cams = plane_scene(logit)
    E = np.array([0.7, 0.8, 0.9])
    albedo = K.sigmoid(np.float32(logit))
    grid = kns.Grid.load(ctx, desc, w)
    try:
        for depth, per_hit in ((1, np.zeros(3)), (2, albedo * E), (4, albedo * E)):
            ref = oracle.path_trace(desc, w, None, cams, 12, 10, 3, depth, 128, 1e-4, 1e-2, 9, E, E)
            got = kns.path_trace(ctx, grid, cams, 12, 10, spp=3, max_depth=depth, seed=9, horizon=E,
                                 zenith=E).cpu().numpy()
            # every path returns E (miss) or per_hit; pixels are means of those values
            np.testing.assert_allclose(got, ref["rgb"], atol=2e-6)
            frac_hit = (ref["traces"] >= 2).mean(1) if depth > 1 else (np.abs(ref["L"]).sum(-1) == 0).mean(1)
            np.testing.assert_allclose(got, (1 - frac_hit)[:, None] * E + frac_hit[:, None] * per_hit, atol=2e-6)
    finally:
        grid.free()


def test_path_trace_matches_oracle_on_the_near_sphere(kns, ctx):
    desc = S.config_desc("c2")
    w = S.sal_sphere_grid(desc, seed=0)
    grid = kns.Grid.load(ctx, desc, w)
    try:
        occ = grid.occupancy()
        cams = S.orbit_cameras(2, 24, 20, seed=7)
        h, z = np.array([1.0, 1.0, 1.0]), np.array([0.5, 0.7, 1.0])
        ref = oracle.path_trace(desc, w, occ, cams, 24, 20, 4, 3, 128, 1e-4, 1e-2, 21, h, z)
        got = kns.path_trace(ctx, grid, cams, 24, 20, spp=4, max_depth=3, seed=21, horizon=h,
                             zenith=z).cpu().numpy()
        err = np.abs(got - ref["rgb"]).max(1)
        # paths are chaotic only where a bounce grazes the surface: almost every pixel agrees closely
        assert np.mean(err <= 2e-4) >= 0.97, np.percentile(err, [50, 90, 99, 100])
        assert np.mean(err) < 5e-3
        # the near-sphere is convex: a bounce never meets it again
        assert (ref["traces"] == 2).any() and ref["traces"].max() == 2
        # deterministic in the seed; a different seed changes the image
        again = kns.path_trace(ctx, grid, cams, 24, 20, spp=4, max_depth=3, seed=21, horizon=h, zenith=z)
        assert np.array_equal(again.cpu().numpy(), got)
        other = kns.path_trace(ctx, grid, cams, 24, 20, spp=4, max_depth=3, seed=22, horizon=h, zenith=z)
        assert not np.array_equal(other.cpu().numpy(), got)
        with pytest.raises(kns.KnsError):
            kns.path_trace(ctx, grid, cams, 24, 20, spp=0)
        with pytest.raises(kns.KnsError):
            kns.path_trace(ctx, grid, cams, 24, 20, max_depth=17)
    finally:
        grid.free()


def two_planes(desc):
    """Floor z = -0.5 in the lower cells, ceiling z = 0.5 in the upper cells (normals facing inwards)."""
    floor = K.plane_grid(desc, [0.0, 0.0, 1.0], 0.5).reshape(desc.n_cells, desc.p_cell)
    ceil = K.plane_grid(desc, [0.0, 0.0, -1.0], 0.5).reshape(desc.n_cells, desc.p_cell)
    iz = np.arange(desc.n_cells) // (desc.N * desc.N)
    w = np.where((iz < desc.N // 2)[:, None], floor, ceil).reshape(-1)
    return K.set_colour_linear(desc, w, [15, 16, 17], [[0.3, 0.0, 0.2], [0.0, 0.4, 0.1], [0.2, 0.1, -0.3]],
                               [0.5, 0.2, 0.9])


def test_path_trace_multiple_bounces(kns, ctx):
    """Between two facing planes paths bounce several times before they leave through a side."""
    desc = S.GridDesc(N=2, sdf_hidden=2, sdf_width=32, col_hidden=1, col_width=32, occ_res=0)
    w = two_planes(desc)
    cams = np.stack([S.look_at_camera([2.5, 0.3, 0.1], 20, 16), S.look_at_camera([-0.4, 2.4, -0.2], 20, 16)])
    h, z = np.array([1.0, 0.95, 0.9]), np.array([0.4, 0.6, 1.0])
    grid = kns.Grid.load(ctx, desc, w)
    try:
        ref = oracle.path_trace(desc, w, None, cams, 20, 16, 4, 6, 128, 1e-4, 1e-2, 5, h, z)
        got = kns.path_trace(ctx, grid, cams, 20, 16, spp=4, max_depth=6, seed=5, horizon=h, zenith=z).cpu().numpy()
        assert (ref["traces"] >= 4).any()
        err = np.abs(got - ref["rgb"]).max(1)
        assert np.mean(err <= 2e-4) >= 0.95, np.percentile(err, [50, 90, 99, 100])
        assert np.mean(err) < 5e-3
    finally:
        grid.free()
