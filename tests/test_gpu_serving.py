"""Multi-view batching and the continuous-batching render server (needs a GPU).

A request's pixels must be the same whether it is rendered alone (kns_render) or inside a batch of
requests of mixed resolutions (kns_render_views, the server): each ray's arithmetic is independent
of the batch, so the results are identical bit for bit."""
import numpy as np
import pytest

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


def solo(kns, ctx, grid, cam, W, H, **kw):
    t = kns.render(ctx, grid, cam[None], W, H, 128, 1e-4, **kw)
    ctx.sync()
    return {k: v.cpu().numpy() for k, v in t.items()}


@pytest.mark.parametrize("precision", [0, 1])
def test_views_batch_equals_solo_renders(kns, precision):
    desc = S.config_desc("c2")
    w = S.sal_sphere_grid(desc)
    ctx = kns.Context(0)
    grid = kns.Grid.load(ctx, desc, w)
    try:
        sizes = [(64, 48), (131, 77), (1, 1), (0, 5), (200, 160), (17, 240)]
        reqs = [(S.orbit_cameras(1, W, H, seed=30 + i)[0], W, H) for i, (W, H) in enumerate(sizes)]
        got = kns.render_views(ctx, grid, reqs, 128, 1e-4, precision=precision)
        ctx.sync()
        for (cam, W, H), t in zip(reqs, got):
            if W * H == 0:
                continue
            ref = solo(kns, ctx, grid, cam, W, H, precision=precision)
            for k in ref:
                assert np.array_equal(ref[k], t[k].cpu().numpy()), (W, H, k)
    finally:
        grid.free()
        ctx.close()


def test_server_mixed_stream_matches_solo(kns):
    from paper_2206_10885_gb300 import serve
    grids = {}
    for name, seed in (("a", 0), ("b", 7)):
        desc = S.config_desc("c2")
        grids[name] = (desc, S.sal_sphere_grid(desc, seed=seed))
    server = serve.RenderServer(grids, slots=2, budget_bytes=64 << 20, max_batch_rays=200_000)
    try:
        stream = serve.poisson_stream(40, rate=2000.0, seed=5, grids=["a", "b"],
                                      resolutions=[(64, 64), (96, 80), (160, 120)])
        stats = serve.run_stream(server, stream)
        assert stats["requests"] == 40 and stats["p99_ms"] >= stats["p50_ms"] > 0
        assert stats["batches"] < 40  # requests were batched
        ctx = kns.Context(0)
        try:
            for _, r in stream:
                ref = solo(kns, ctx, server.grids[r.grid], r.cam, r.W, r.H)
                for k in ref:
                    assert np.array_equal(ref[k], r.out[k].cpu().numpy()), (r.rid, k)
        finally:
            ctx.close()
    finally:
        server.close()
