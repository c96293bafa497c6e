"""Failure path of the bounded device waits (needs a GPU; nothing faults, traps or hangs).

Every wait in the render's kernels -- the mbarrier waits of the tensor-core tiles (weights, products)
and the persistent trace's grid barrier -- gives up after a poll limit, records KNS_ERR_TIMEOUT in the
context's status word and returns.  kns_selftest_timeout runs such a wait that nothing satisfies (an
mbarrier no thread arrives at; a grid barrier one of two blocks never reaches) with a short limit.
The test checks that the next kns_sync reports KNS_ERR_TIMEOUT, that the status is cleared after it,
and that the same context then renders correctly (against the FP64 oracle, in BF16 and FP32).
"""
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


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_reports_timeout_and_context_recovers(kns, which):
    from paper_2206_10885_gb300 import _capi as capi
    ctx = kns.Context(0)
    try:
        desc = S.config_desc("c2")
        w = S.sal_sphere_grid(desc)
        occ = O.occupancy(desc, w)
        grid = kns.Grid.load(ctx, desc, w, occ)
        cams = S.orbit_cameras(1, 40, 32, seed=5)
        ctx.sync()
        capi.kns_selftest_timeout(ctx.handle, which, 0)
        with pytest.raises(capi.KnsError) as err:
            ctx.sync()
        assert err.value.status == capi.KNS_ERR_TIMEOUT
        ctx.sync()  # the status word was cleared by the report
        o = O.render(desc, w, occ, cams, 40, 32, 128, 1e-4)
        for precision in (kns.KNS_BF16, kns.KNS_FP32):
            t = kns.render(ctx, grid, cams, 40, 32, 128, 1e-4, precision=precision)
            ctx.sync()
            g = {k: v.cpu().numpy() for k, v in t.items()}
            both = (g["hit"] == 1) & (o["hit"] == 1)
            assert np.mean(g["hit"] == o["hit"]) > 0.99
            assert both.sum() > 50
            assert np.mean(np.abs(g["depth"][both] - o["depth"][both]) <= 1e-3) >= 0.999
        grid.free()
    finally:
        ctx.close()


def test_selftest_rejects_unknown_wait(kns):
    from paper_2206_10885_gb300 import _capi as capi
    ctx = kns.Context(0)
    try:
        with pytest.raises(capi.KnsError) as err:
            capi.kns_selftest_timeout(ctx.handle, 2, 0)
        assert err.value.status == capi.KNS_ERR_INVALID_ARG
    finally:
        ctx.close()
