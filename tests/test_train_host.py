"""Host side of the training step (CPU only): the seeded batch draws and the marshalling of a
TrainBatch into the C struct."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2206_10885_gb300 import synth as S

torch = pytest.importorskip("torch")


def test_train_draws_shapes_ranges_and_seeding():
    sel, u_s, u_i, pts = S.train_draws(1000, 64, 32, 500, n_pix=640000, seed=3)
    assert sel.shape == (1000,) and sel.dtype == np.int64 and sel.min() >= 0 and sel.max() < 640000
    assert u_s.shape == (1000, 64) and u_s.dtype == np.float32 and u_s.min() >= 0 and u_s.max() < 1
    assert u_i.shape == (1000, 32) and np.all(np.diff(u_i, axis=1) >= 0)     # importance uniforms ascend
    assert pts.shape == (500, 3) and pts.min() >= -1 and pts.max() <= 1
    again = S.train_draws(1000, 64, 32, 500, n_pix=640000, seed=3)
    assert all(np.array_equal(a, b) for a, b in zip((sel, u_s, u_i, pts), again))
    other = S.train_draws(1000, 64, 32, 500, n_pix=640000, seed=4)
    assert not np.array_equal(u_s, other[1])
    assert abs(u_s.mean() - 0.5) < 0.01 and abs(pts.mean()) < 0.05


def test_train_batch_marshalling():
    from paper_2206_10885_gb300 import train as T
    B, Ns, Ni, M = 7, 5, 3, 11
    o = torch.randn(B, 3)
    d = torch.nn.functional.normalize(torch.randn(3, B).t(), dim=1)   # not contiguous
    assert not d.is_contiguous()
    batch = T.TrainBatch(o, d, torch.rand(B, 3), torch.rand(B, Ns), torch.rand(B, Ni).sort(1).values,
                         torch.rand(M, 3) * 2 - 1, s=30.0, s_up=80.0, lam=0.25, h=5e-3, timing=True)
    assert batch.dirs.is_contiguous()
    assert batch.n_rays == B and batch.samples == Ns + Ni
    c = batch.c_struct()
    assert (c.n_rays, c.n_strat, c.n_imp, c.n_eik) == (B, Ns, Ni, M)
    assert c.origins == o.data_ptr() and c.dirs == batch.dirs.data_ptr() and c.target == batch.target.data_ptr()
    assert c.u_strat == batch.u_strat.data_ptr() and c.u_imp == batch.u_imp.data_ptr()
    assert c.eik_points == batch.eik_points.data_ptr() and not c.t_fixed
    assert (c.s, c.s_up, c.h) == pytest.approx((30.0, 80.0, 5e-3)) and c.lambda_ == pytest.approx(0.25)
    assert c.timing == 1
    # empty importance samples and eikonal points pass NULL
    empty = T.TrainBatch(o, d, torch.rand(B, 3), torch.rand(B, Ns), torch.zeros(B, 0), torch.zeros(0, 3),
                         t_fixed=torch.rand(B, Ns))
    c = empty.c_struct()
    assert not c.u_imp and not c.eik_points and c.n_imp == 0 and c.n_eik == 0
    assert c.t_fixed == empty.t_fixed.data_ptr() and c.timing == 0
