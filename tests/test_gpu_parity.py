"""FP32 CUDA path vs the FP64 oracle, element by element, through the C ABI (needs a GPU)."""
import os

import numpy as np
import pytest

import gridkit as K
import oracle as O
import parity as P
from paper_2206_10885_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10885_gb300 import build as kbuild
    kbuild.build()
    import paper_2206_10885_gb300 as kns
    return kns


@pytest.fixture(scope="module")
def ctx(kns):
    c = kns.Context(0)
    yield c
    c.close()


def gpu_render(kns, ctx, grid, cams, W, H, ms, eps, **kw):
    t = kns.render(ctx, grid, cams, W, H, ms, eps, **kw)
    ctx.sync()
    return P.to_np(t)


def sel_rows(d, sel):
    return {k: v[sel] for k, v in d.items()}


# ------------------------------------------------------------------ batch field query
def sdf_compare(kns, ctx, desc, w, pts, tol_d, tol_g):
    grid = kns.Grid.load(ctx, desc, w)
    try:
        d, f, g = kns.sdf(ctx, grid, torch.from_numpy(pts).cuda())
        ctx.sync()
        d, f, g = d.cpu().numpy(), f.cpu().numpy(), g.cpu().numpy()
    finally:
        grid.free()
    od, of, og, _ = O.sdf(desc, w, pts.astype(np.float64))
    scale_g = np.maximum(1.0, np.abs(og))
    assert np.max(np.abs(d - od)) <= tol_d, np.max(np.abs(d - od))
    assert np.max(np.abs(f - of)) <= tol_d, np.max(np.abs(f - of))
    assert np.max(np.abs(g - og) / scale_g) <= tol_g, np.max(np.abs(g - og) / scale_g)
    return np.max(np.abs(d - od))


def test_sdf_sal_grid(kns, ctx):
    desc = S.config_desc("c2")
    w = S.sal_sphere_grid(desc)
    pts = S.uniform_points(20000, seed=3)
    # points exactly on cell faces too (ties go to the higher cell on both sides)
    faces = pts[:500].copy()
    faces[:, 0] = np.round(faces[:, 0] * 8) / 8
    sdf_compare(kns, ctx, desc, w, np.concatenate([pts, faces]), 2e-6, 1e-5)


@pytest.mark.parametrize("width,hidden,L,LD", [(32, 2, 4, 2), (32, 3, 4, 2), (64, 2, 4, 2), (64, 3, 4, 2),
                                               (32, 2, 6, 4), (32, 3, 6, 4), (64, 2, 6, 4), (64, 3, 6, 4)])
def test_sdf_every_config_dense_random(kns, ctx, width, hidden, L, LD):
    desc = S.GridDesc(N=3, sdf_width=width, col_width=width, sdf_hidden=hidden, pe_pos_L=L, pe_dir_L=LD,
                      softplus_beta=10.0)
    w = K.random_grid(desc, seed=width + hidden + L, scale=0.3)
    pts = S.uniform_points(3000, seed=width * hidden)
    sdf_compare(kns, ctx, desc, w, pts, 2e-5, 1e-4)


def test_sdf_plane_is_exact(kns, ctx):
    desc = S.GridDesc(N=4, sdf_hidden=3)
    a = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    w = K.plane_grid(desc, a, 0.1)
    pts = S.uniform_points(5000, seed=9)
    sdf_compare(kns, ctx, desc, w, pts, 1e-6, 1e-6)


def test_sdf_empty_and_ragged(kns, ctx):
    desc = S.config_desc("c1")
    w = S.sal_sphere_grid(desc)
    grid = kns.Grid.load(ctx, desc, w)
    try:
        d, _, _ = kns.sdf(ctx, grid, torch.zeros((0, 3), device="cuda"))
        assert d.numel() == 0
        pts = S.uniform_points(129, seed=1)  # one full block plus a ragged tail of one
        d, _, _ = kns.sdf(ctx, grid, torch.from_numpy(pts).cuda())
        ctx.sync()
        od, _, _, _ = O.sdf(desc, w, pts.astype(np.float64))
        assert np.max(np.abs(d.cpu().numpy() - od)) < 2e-6
    finally:
        grid.free()


# ------------------------------------------------------------------ occupancy builder
def test_occupancy_builder_matches_oracle(kns, ctx):
    desc = S.config_desc("c2")
    w = S.sal_sphere_grid(desc)
    grid = kns.Grid.load(ctx, desc, w)  # no mask given: built on the device
    try:
        got = np.unpackbits(grid.occupancy().view(np.uint8), bitorder="little").astype(bool)
    finally:
        grid.free()
    want = np.unpackbits(O.occupancy(desc, w).view(np.uint8), bitorder="little").astype(bool)
    diff = np.where(got != want)[0]
    if diff.size:
        res = desc.occ_res
        ix, iy, iz = diff % res, (diff // res) % res, diff // (res * res)
        c = -1 + (np.stack([ix, iy, iz], 1) + 0.5) * (2 / res)
        d, _, _, _ = O.sdf(desc, w, c)
        diag = np.sqrt(3) * 2 / res
        assert np.all(np.abs(np.abs(d) - diag) < 1e-5), np.abs(np.abs(d) - diag).max()
    assert want.sum() > 1000 and diff.size <= 10


# ------------------------------------------------------------------ render
def test_render_c1_full(kns, ctx):
    desc, w, cams, W, H, ms, eps = S.workload("c1")
    grid = kns.Grid.load(ctx, desc, w)
    try:
        g = gpu_render(kns, ctx, grid, cams, W, H, ms, eps)
    finally:
        grid.free()
    o = O.render(desc, w, None, cams, W, H, ms, eps, delta_step=P.DELTA_STEP)
    s = P.compare_render(g, o, label="c1", min_robust=0.94)
    assert s["hits"] > 2000


def test_render_occupancy_ragged(kns, ctx):
    """16^3 grid with the 128^3 mask (the oracle's), 2 cameras at 120x100 (ragged tiles)."""
    desc = S.config_desc("c2")
    w = S.sal_sphere_grid(desc)
    occ = O.occupancy(desc, w)
    cams = S.orbit_cameras(2, 120, 100, seed=5)
    grid = kns.Grid.load(ctx, desc, w, occ)
    try:
        g = gpu_render(kns, ctx, grid, cams, 120, 100, 128, 1e-4)
    finally:
        grid.free()
    o = O.render(desc, w, occ, cams, 120, 100, 128, 1e-4, delta_step=P.DELTA_STEP)
    s = P.compare_render(g, o, label="occ", min_robust=0.85)
    assert s["hits"] > 2000


def test_render_c3l_launch_sampled(kns, ctx):
    """The 1080p launch the benchmark times (8 cameras x 1920x1080, 32^3 grid of width 64, mask, 128 steps)
    in FP32, on sampled rays: the FP32 gates."""
    desc, w, cams, W, H, ms, eps = S.workload("c3l")
    occ = O.occupancy(desc, w)
    grid = kns.Grid.load(ctx, desc, w, occ)
    try:
        g = gpu_render(kns, ctx, grid, cams, W, H, ms, eps)
    finally:
        grid.free()
    rng = np.random.default_rng(1)
    n_pix = cams.shape[0] * W * H
    sel = np.unique(np.concatenate([rng.integers(0, n_pix, 2000),
                                    np.where(g["hit"] == 1)[0][rng.integers(0, int(g["hit"].sum()), 2000)]]))
    o = O.render(desc, w, occ, cams, W, H, ms, eps, sel=sel, delta_step=P.DELTA_STEP)
    s = P.compare_render(sel_rows(g, sel), o, label="c3l-sampled", min_robust=0.8)
    assert s["hits"] > 1500


def test_render_full_size_sampled(kns, ctx):
    """The benchmark's launch: 8 cameras x 800x800, 16^3 grid, mask, 128 steps; sampled rays."""
    desc, w, cams, W, H, ms, eps = S.workload("c2")
    occ = O.occupancy(desc, w)
    grid = kns.Grid.load(ctx, desc, w, occ)
    try:
        g = gpu_render(kns, ctx, grid, cams, W, H, ms, eps)
    finally:
        grid.free()
    rng = np.random.default_rng(0)
    n_pix = cams.shape[0] * W * H
    sel = np.unique(np.concatenate([rng.integers(0, n_pix, 3000),
                                    np.where(g["hit"] == 1)[0][rng.integers(0, int(g["hit"].sum()), 3000)]]))
    o = O.render(desc, w, occ, cams, W, H, ms, eps, sel=sel, delta_step=P.DELTA_STEP)
    s = P.compare_render(sel_rows(g, sel), o, label="c2-sampled", min_robust=0.84)
    assert s["hits"] > 2500
    # whole-image invariants: every hit has a unit normal and depth inside the box interval
    h = g["hit"] == 1
    assert np.allclose(np.linalg.norm(g["normal"][h], axis=1), 1.0, atol=1e-5)
    assert np.all(g["depth"][h] > 0) and np.all(g["depth"][h] < 2.5 + 2 * np.sqrt(3))


def test_render_plane_cell_colours(kns, ctx):
    """Exact plane with per-cell colour biases: cells and colours identify the hit cell."""
    desc = S.GridDesc(N=8, sdf_hidden=2)
    a = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    cb = np.zeros((desc.n_cells, 3))
    ids = np.arange(desc.n_cells)
    cb[:, 0], cb[:, 1], cb[:, 2] = (ids % 8) * 0.25 - 1, ((ids // 8) % 8) * 0.25 - 1, (ids // 64) * 0.25 - 1
    w = K.set_colour_linear(desc, K.plane_grid(desc, a, 0.1), [0], np.zeros((3, 1)), [0, 0, 0], cell_bias=cb)
    cams = K.plane_side_cameras(a, 3, 64, 48, seed=7)
    grid = kns.Grid.load(ctx, desc, w)
    try:
        g = gpu_render(kns, ctx, grid, cams, 64, 48, 64, 1e-4)
    finally:
        grid.free()
    o = O.render(desc, w, None, cams, 64, 48, 64, 1e-4, delta_step=P.DELTA_STEP)
    # an exact plane converges geometrically, so many steps land close to |d| = eps: every robust
    # ray must agree exactly; the non-robust remainder may flip
    s = P.compare_render(g, o, min_agree=0.995, label="plane", min_robust=0.94)
    assert s["hits"] > 1000


def test_render_linear_colour_routes_normal_and_view(kns, ctx):
    desc = S.GridDesc(N=4, sdf_hidden=3)
    a = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    rng = np.random.default_rng(2)
    F = desc.feat_dim
    w = K.plane_grid(desc, a, 0.1, feat_c=rng.uniform(-1, 1, F), feat_e=rng.uniform(-1, 1, F))
    sel = [0, 14, F, F + 1, F + 2, F + 3, F + 4, F + 5, F + 6, F + 3 + 14]
    w = K.set_colour_linear(desc, w, sel, rng.uniform(-1, 1, (3, len(sel))), rng.uniform(-0.5, 0.5, 3))
    cams = K.plane_side_cameras(a, 2, 40, 40, seed=11)
    grid = kns.Grid.load(ctx, desc, w)
    try:
        g = gpu_render(kns, ctx, grid, cams, 40, 40, 64, 1e-5)
    finally:
        grid.free()
    o = O.render(desc, w, None, cams, 40, 40, 64, 1e-5, delta_step=P.DELTA_STEP)
    s = P.compare_render(g, o, label="linear-colour", min_robust=0.6)
    assert s["hits"] > 1000


@pytest.mark.parametrize("width,hidden,L,LD", [(32, 2, 4, 2), (64, 3, 4, 2), (32, 3, 6, 4), (64, 2, 6, 4)])
def test_render_other_configs(kns, ctx, width, hidden, L, LD):
    desc = S.GridDesc(N=8, sdf_width=width, col_width=width, sdf_hidden=hidden, pe_pos_L=L, pe_dir_L=LD,
                      occ_res=64)
    w = S.sal_sphere_grid(desc, seed=4)
    occ = O.occupancy(desc, w)
    cams = S.orbit_cameras(2, 48, 40, seed=2)
    grid = kns.Grid.load(ctx, desc, w, occ)
    try:
        g = gpu_render(kns, ctx, grid, cams, 48, 40, 96, 1e-4)
    finally:
        grid.free()
    o = O.render(desc, w, occ, cams, 48, 40, 96, 1e-4, delta_step=P.DELTA_STEP)
    P.compare_render(g, o, min_agree=0.995, label=str((width, hidden, L, LD)), min_robust=0.83)


def test_render_edge_cases(kns, ctx):
    desc, w, cams, W, H, ms, eps = S.workload("c1")
    grid = kns.Grid.load(ctx, desc, w)
    try:
        # empty launches are successful no-ops
        t = kns.alloc_frame(1)
        kns.capi.kns_render(ctx.handle, grid.handle, cams.ctypes.data, 0, 64, 64, 64, 1e-4, None, t[1], 0)
        kns.capi.kns_render(ctx.handle, grid.handle, cams.ctypes.data, 1, 0, 64, 64, 1e-4, None, t[1], 0)
        # 1x1 image, one-step budget, a camera inside the box, and more cameras than one launch takes
        inside = S.look_at_camera([0.2, 0.1, 0.9], 16, 16)
        many = S.orbit_cameras(70, 8, 6, seed=9)
        for cams_, W_, H_, ms_ in [(cams[:1], 1, 1, 64), (cams[:2], 17, 9, 1), (inside[None], 16, 16, 64),
                                   (many, 8, 6, 64)]:
            g = gpu_render(kns, ctx, grid, cams_, W_, H_, ms_, eps)
            o = O.render(desc, w, None, cams_, W_, H_, ms_, eps, delta_step=P.DELTA_STEP)
            P.compare_render(g, o, min_agree=0.99, label=str((W_, H_, ms_)))
    finally:
        grid.free()


def test_render_rejects_bad_arguments(kns, ctx):
    desc, w, cams, W, H, ms, eps = S.workload("c1")
    grid = kns.Grid.load(ctx, desc, w)
    capi = kns.capi
    t, f = kns.alloc_frame(64 * 64)
    try:
        for args, code in [((1, 64, 64, 0, 1e-4), capi.KNS_ERR_INVALID_ARG),
                           ((1, 64, 64, 8, 0.0), capi.KNS_ERR_INVALID_ARG),
                           ((1, 64, 64, 8, float("nan")), capi.KNS_ERR_INVALID_ARG),
                           ((-1, 64, 64, 8, 1e-4), capi.KNS_ERR_INVALID_ARG),
                           ((1 << 20, 1 << 20, 1 << 10, 8, 1e-4), capi.KNS_ERR_INVALID_ARG)]:
            with pytest.raises(capi.KnsError) as e:
                capi.kns_render(ctx.handle, grid.handle, cams.ctypes.data, *args, None, f, 0)
            assert e.value.status == code
        bad = capi.kns_frame()
        with pytest.raises(capi.KnsError) as e:
            capi.kns_render(ctx.handle, grid.handle, cams.ctypes.data, 1, 8, 8, 8, 1e-4, None, bad, 0)
        assert e.value.status == capi.KNS_ERR_INVALID_ARG
        with pytest.raises(capi.KnsError) as e:
            capi.kns_load_grid(ctx.handle, desc, w.ctypes.data, w.size - 1)
        assert e.value.status == capi.KNS_ERR_INVALID_ARG
        odd = S.GridDesc(N=4, sdf_width=48, col_width=48)
        with pytest.raises(capi.KnsError) as e:
            capi.kns_load_grid(ctx.handle, odd, w.ctypes.data, odd.n_cells * odd.p_cell)
        assert e.value.status == capi.KNS_ERR_UNSUPPORTED
        ctx.sync()
    finally:
        grid.free()


def test_grid_file_roundtrip(kns, ctx, tmp_path):
    desc = S.config_desc("c2")
    w = S.sal_sphere_grid(desc)
    occ = O.occupancy(desc, w)
    path = str(tmp_path / "g.kns")
    S.write_kns(path, desc, w, occ)
    cams = S.orbit_cameras(1, 64, 64, seed=3)
    g1 = kns.Grid.load(ctx, desc, w, occ)
    g2 = kns.Grid.from_file(ctx, path)
    try:
        a = gpu_render(kns, ctx, g1, cams, 64, 64, 128, 1e-4)
        b = gpu_render(kns, ctx, g2, cams, 64, 64, 128, 1e-4)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    finally:
        g1.free()
        g2.free()
    with open(path, "r+b") as fh:
        fh.write(b"XXXX")
    with pytest.raises(kns.KnsError) as e:
        kns.Grid.from_file(ctx, path)
    assert e.value.status == kns.capi.KNS_ERR_FORMAT


def test_schedule_knobs_do_not_change_results(kns, ctx):
    """The tuning fields of kns_render_opts reorder work only: every output is bit-identical."""
    desc = S.config_desc("c2")
    w = S.sal_sphere_grid(desc)
    cams = S.orbit_cameras(2, 160, 120, seed=8)
    grid = kns.Grid.load(ctx, desc, w)
    try:
        ref = gpu_render(kns, ctx, grid, cams, 160, 120, 128, 1e-4)
        for tuning in [dict(block_tiles=2, inner_steps=1, min_active=1, static_tiles=2, tail_rays=-1),
                       dict(block_tiles=2, inner_steps=64, min_active=16, static_tiles=1, blocks_per_sm=2,
                            tail_rays=4096),
                       dict(block_tiles=2, inner_steps=7, min_active=3, static_tiles=2, blocks_per_sm=16,
                            tail_rays=100000),
                       dict(block_tiles=1, static_tiles=1, tail_rays=-1),
                       dict(block_tiles=3, static_tiles=2, tail_rays=4096),
                       dict(block_tiles=3, static_tiles=1, tail_rays=-1),
                       dict(block_tiles=4, static_tiles=2, tail_rays=-1),
                       dict(block_tiles=1, inner_steps=4, min_active=1, tail_rays=-1),
                       dict(block_tiles=4, inner_steps=3, min_active=40, tail_rays=4096),
                       dict(block_tiles=3, inner_steps=128, min_active=1, static_tiles=1, tail_rays=-1)]:
            got = gpu_render(kns, ctx, grid, cams, 160, 120, 128, 1e-4, tuning=tuning)
            for k in ref:
                assert np.array_equal(ref[k], got[k]), (k, tuning)
        with pytest.raises(kns.KnsError):
            kns.render(ctx, grid, cams, 160, 120, 128, 1e-4, tuning=dict(min_active=257))
        with pytest.raises(kns.KnsError):
            kns.render(ctx, grid, cams, 160, 120, 128, 1e-4, tuning=dict(block_tiles=5))
    finally:
        grid.free()
