"""kns_render_noalloc: the allocation-free render for callers that may not allocate device memory
while running (an application whose device memory all belongs to its own pool allocator, or a
latency-bound loop that cannot take cudaMalloc's implicit synchronisation).  It must give the same
pixels as kns_render, call after call, from its built-in scratch.  This file is collected last so
that a failure here comes after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_render_matches_kns_render_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10885_gb300 import build as kbuild
    kbuild.build()
    import paper_2206_10885_gb300 as kns
    from paper_2206_10885_gb300 import synth as S

    desc = S.config_desc("c2")
    w = S.sal_sphere_grid(desc)
    cams = S.orbit_cameras(2, 320, 240, seed=3)  # 153,600 rays: inside the built-in limit
    ctx = kns.Context(0)
    grid = kns.Grid.load(ctx, desc, w)
    try:
        ref = kns.render(ctx, grid, cams, 320, 240, 128, 1e-4)
        ctx.sync()
        ref = {k: v.cpu().numpy() for k, v in ref.items()}
        for call in range(2):
            t, f = kns.alloc_frame(cams.shape[0] * 320 * 240)
            for v in t.values():  # stale contents must not survive into the result
                v.fill_(7)
            kns.capi.kns_render_noalloc(ctx.handle, grid.handle, cams.ctypes.data, cams.shape[0], 320, 240, 128,
                                        1e-4, f, torch.cuda.current_stream().cuda_stream)
            ctx.sync()
            got = {k: v.cpu().numpy() for k, v in t.items()}
            for k in ref:
                if ref[k].dtype.kind == "f":
                    both_inf = np.isinf(ref[k]) & np.isinf(got[k])
                    fin = ~both_inf
                    assert np.all(np.isfinite(got[k][fin])), (call, k)
                    assert np.all(np.abs(ref[k][fin] - got[k][fin]) <= 1e-6), (call, k)
                else:
                    assert np.array_equal(ref[k], got[k]), (call, k)
        # beyond the built-in scratch: a clear argument error, nothing enqueued
        big = S.orbit_cameras(1, 1024, 1024, seed=3)
        t, f = kns.alloc_frame(1024 * 1024, extras=False)
        with pytest.raises(kns.KnsError) as e:
            kns.capi.kns_render_noalloc(ctx.handle, grid.handle, big.ctypes.data, 1, 1024, 1024, 128, 1e-4, f,
                                        torch.cuda.current_stream().cuda_stream)
        assert e.value.status == kns.capi.KNS_ERR_INVALID_ARG and "limit" in str(e.value)
        ctx.sync()
    finally:
        grid.free()
        ctx.close()
