"""Multi-view batching and the continuous-batching render server (needs a GPU).

A request's pixels must be the same whether it is rendered alone (kns_render) or inside a batch of
requests of mixed resolutions (kns_render_views, the server).  In FP32 each ray's arithmetic is
independent of the batch, so the results are identical bit for bit.  In BF16 the batch decides which
of a ray's last steps run in FP32 (the one-warp-per-ray tail of small rounds), so the results agree
within the BF16 accuracy gates -- and both agree with the FP64 oracle within them."""
import numpy as np
import pytest

import oracle as O
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


def assert_within_bf16_gates(a, b, label):
    """Two BF16 renders of the same pixels: hit agreement and, on pixels both hit, depth within 1e-3,
    RGB within 1/255 and normal angle within 0.5 degrees, each on >= 99.9 % of pixels."""
    ha, hb = a["hit"] == 1, b["hit"] == 1
    both = ha & hb
    n = max(1, ha.size)
    assert np.sum(ha != hb) <= max(1, int(1e-3 * n)), (label, "hit agreement", int(np.sum(ha != hb)), n)
    if both.sum() == 0:
        return
    dd = np.abs(a["depth"][both].astype(np.float64) - b["depth"][both])
    dr = np.abs(a["rgb"][both].astype(np.float64) - b["rgb"][both]).max(axis=1)
    ang = np.degrees(np.arccos(np.clip(np.sum(a["normal"][both].astype(np.float64) * b["normal"][both], axis=1), -1, 1)))
    k = max(1, int(1e-3 * both.sum()))  # at most 0.1 % of both-hit pixels outside each gate
    assert np.sum(dd > 1e-3) <= k and np.sum(dr > 1 / 255) <= k and np.sum(ang > 0.5) <= k, (label, dd.max(), dr.max(),
                                                                                            ang.max())


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
            got = {k: v.cpu().numpy() for k, v in t.items()}
            if precision == kns.KNS_FP32:  # the FP32 path is schedule-invariant: identical bit for bit
                for k in ref:
                    assert np.array_equal(ref[k], got[k]), (W, H, k)
            else:  # BF16: the batch decides which last steps run in FP32; results agree within the gates
                assert_within_bf16_gates(ref, got, (W, H))
    finally:
        grid.free()
        ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_stack_views_equal_grids_alone(kns, precision):
    """Three grids of one shape loaded as a stack: a batch of views of all three renders every view as
    the grid loaded alone renders it (FP32 bit for bit, BF16 within the gates), each grid keeps its own
    occupancy mask, and a view naming a grid outside the stack is refused."""
    desc = S.config_desc("c2")
    ws = [S.sal_sphere_grid(desc, seed=s) for s in (0, 7, 11)]
    ctx = kns.Context(0)
    stack = kns.Grid.load_stack(ctx, desc, ws)
    alone = [kns.Grid.load(ctx, desc, w) for w in ws]
    try:
        assert stack.n_grids == 3 and alone[0].n_grids == 1
        occ_stack = stack.occupancy()
        per = occ_stack.size // 3
        for k in range(3):
            assert np.array_equal(occ_stack[k * per:(k + 1) * per], alone[k].occupancy()), k
        sizes = [(64, 48, 2), (131, 77, 0), (1, 1, 1), (0, 5, 2), (200, 160, 1), (17, 240, 0), (96, 96, 2)]
        reqs = [(S.orbit_cameras(1, W, H, seed=40 + i)[0], W, H, k) for i, (W, H, k) in enumerate(sizes)]
        got = kns.render_views(ctx, stack, reqs, 128, 1e-4, precision=precision)
        ctx.sync()
        for (cam, W, H, k), t in zip(reqs, got):
            if W * H == 0:
                continue
            ref = solo(kns, ctx, alone[k], cam, W, H, precision=precision)
            g = {key: v.cpu().numpy() for key, v in t.items()}
            if precision == kns.KNS_FP32:
                for key in ref:
                    assert np.array_equal(ref[key], g[key]), (W, H, k, key)
            else:
                assert_within_bf16_gates(ref, g, (W, H, k))
        # the stack's grids differ: the same view of two grids is not the same image
        a, b = kns.render_views(ctx, stack, [(reqs[0][0], 64, 48, 0), (reqs[0][0], 64, 48, 1)], 128, 1e-4,
                                precision=precision)
        ctx.sync()
        assert not np.array_equal(a["depth"].cpu().numpy(), b["depth"].cpu().numpy())
        with pytest.raises(kns.KnsError):
            kns.render_views(ctx, stack, [(reqs[0][0], 8, 8, 3)], 128, 1e-4, precision=precision)
    finally:
        for g in alone:
            g.free()
        stack.free()
        ctx.close()


def test_server_mixed_stream_matches_solo(kns):
    """Two grids of one shape: the server stacks them, batches requests for both into one launch
    sequence, and every request equals its grid's solo render (loaded alone) bit for bit."""
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
        assert stats["mixed_batches"] > 0, stats  # and batches held requests for both grids
        ctx = kns.Context(0)
        alone = {name: kns.Grid.load(ctx, d, w) for name, (d, w) in grids.items()}
        try:
            for _, r in stream:
                ref = solo(kns, ctx, alone[r.grid], r.cam, r.W, r.H)
                for k in ref:
                    assert np.array_equal(ref[k], r.out[k].cpu().numpy()), (r.rid, k)
        finally:
            for g in alone.values():
                g.free()
            ctx.close()
    finally:
        server.close()


def test_server_bf16_mixed_stream_matches_oracle(kns):
    """BF16 serving of two 16^3 width-32 grids (one stack) and a 32^3 width-64 grid (the workload's two grid
    shapes): sampled pixels of every request of a mixed stream against the FP64 oracle, within the BF16 gates
    (depth 1e-3, RGB 1/255, normal 0.5 degrees on >= 99.9 % of pixels both hit; hit agreement >= 99.9 %)."""
    from paper_2206_10885_gb300 import serve
    grids = {"s": (S.config_desc("c3s"), S.sal_sphere_grid(S.config_desc("c3s"), seed=0)),
             "t": (S.config_desc("c3s"), S.sal_sphere_grid(S.config_desc("c3s"), seed=1)),
             "l": (S.config_desc("c3l"), S.sal_sphere_grid(S.config_desc("c3l"), seed=0))}
    occs = {k: O.occupancy(d, w) for k, (d, w) in grids.items()}
    server = serve.RenderServer({k: (d, w, occs[k]) for k, (d, w) in grids.items()}, slots=2,
                                budget_bytes=256 << 20, max_batch_rays=400_000, precision=kns.KNS_BF16)
    try:
        stream = serve.poisson_stream(15, rate=500.0, seed=9, grids=["s", "t", "l"],
                                      resolutions=[(64, 64), (160, 120), (256, 256)])
        stats = serve.run_stream(server, stream)
        assert stats["requests"] == 15
        rng = np.random.default_rng(3)
        tot = agree = 0
        bad = {"depth": 0, "rgb": 0, "normal": 0}
        both_n = 0
        for _, r in stream:
            desc, w = grids[r.grid]
            g = {k: v.cpu().numpy() for k, v in r.out.items()}
            sel = np.unique(rng.integers(0, r.W * r.H, 400))
            o = O.render(desc, w, occs[r.grid], r.cam[None], r.W, r.H, 128, 1e-4, sel=sel)
            gs = {k: v[sel] for k, v in g.items()}
            gh, oh = gs["hit"] == 1, o["hit"] == 1
            tot += sel.size
            agree += int(np.sum(gh == oh))
            both = gh & oh
            both_n += int(both.sum())
            bad["depth"] += int(np.sum(np.abs(gs["depth"][both] - o["depth"][both]) > 1e-3))
            bad["rgb"] += int(np.sum(np.abs(gs["rgb"][both] - o["rgb"][both]).max(axis=1) > 1 / 255))
            cosang = np.clip(np.sum(gs["normal"][both] * o["normal"][both], axis=1), -1, 1)
            bad["normal"] += int(np.sum(np.degrees(np.arccos(cosang)) > 0.5))
        print("bf16 serving vs oracle: pixels", tot, "hit agreement", agree / tot, "both", both_n, bad)
        assert agree >= 0.999 * tot
        assert both_n > 300
        assert all(v <= 1e-3 * both_n for v in bad.values()), bad
    finally:
        server.close()
