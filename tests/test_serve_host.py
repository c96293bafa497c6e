"""Host logic of the render server (CPU only): batch formation under the HBM budget and the ray cap,
and the seeded Poisson request stream."""
from __future__ import annotations

import collections
import threading

import numpy as np

from paper_2206_10885_gb300 import serve as SV


def bare_server(budget, max_rays):
    """A RenderServer without device slots: only the scheduling state _take_batch reads."""
    s = SV.RenderServer.__new__(SV.RenderServer)
    s.pending = collections.deque()
    s.budget = budget
    s.max_batch_rays = max_rays
    s.in_flight_bytes = 0
    s.in_flight = 0
    s.batches = 0
    s.mixed_batches = 0
    s.cv = threading.Condition()
    return s


def req(rid, grid, W, H):
    return SV.Request(rid, grid, np.zeros(16, np.float32), W, H)


def test_batch_takes_the_oldest_grid_in_order_up_to_the_ray_cap():
    s = bare_server(budget=1 << 40, max_rays=3 * 100 * 100)
    rs = [req(0, "a", 100, 100), req(1, "b", 100, 100), req(2, "a", 100, 100), req(3, "a", 100, 100),
          req(4, "a", 100, 100), req(5, "b", 50, 50)]
    s.pending.extend(rs)
    g, take = s._take_batch()
    assert g == "a" and [r.rid for r in take] == [0, 2, 3]          # the cap stops at three 100^2 views
    assert [r.rid for r in s.pending] == [1, 4, 5]                  # the rest keep their order
    assert s.in_flight == 1 and s.batches == 1
    assert s.in_flight_bytes == sum(r.bytes for r in take)
    g, take = s._take_batch()
    assert g == "b" and [r.rid for r in take] == [1, 5]
    g, take = s._take_batch()
    assert g == "a" and [r.rid for r in take] == [4]
    assert s._take_batch() == (None, [])
    assert s.batches == 3


def test_batch_spans_the_grids_of_one_stack():
    """Grids loaded as one stack (equal descriptors) share batches: the oldest request's stack decides,
    and every admitted request for any of its grids joins, in order."""
    s = bare_server(budget=1 << 40, max_rays=1 << 30)
    s.group_of = {"a": "k32", "b": "k32", "c": "k64"}
    s.pending.extend([req(0, "a", 64, 64), req(1, "c", 64, 64), req(2, "b", 64, 64), req(3, "a", 32, 32),
                      req(4, "c", 16, 16)])
    key, take = s._take_batch()
    assert key == "k32" and [r.rid for r in take] == [0, 2, 3]
    assert s.mixed_batches == 1
    key, take = s._take_batch()
    assert key == "k64" and [r.rid for r in take] == [1, 4]
    assert s.mixed_batches == 1 and s.batches == 2


def test_grids_stack_by_descriptor():
    from paper_2206_10885_gb300 import synth as S
    a, b, c = S.config_desc("c3s"), S.config_desc("c2"), S.config_desc("c3l")
    assert SV.desc_key(a) == SV.desc_key(b)      # same shape: one stack
    assert SV.desc_key(a) != SV.desc_key(c)      # another width and N: a stack of its own


def test_a_request_larger_than_the_cap_goes_alone():
    s = bare_server(budget=1 << 40, max_rays=1000)
    s.pending.extend([req(0, "a", 1920, 1080), req(1, "a", 10, 10)])
    _, take = s._take_batch()
    assert [r.rid for r in take] == [0]
    _, take = s._take_batch()
    assert [r.rid for r in take] == [1]


def test_admission_by_hbm_budget():
    one = req(0, "a", 100, 100).bytes
    s = bare_server(budget=2 * one, max_rays=1 << 30)
    s.pending.extend([req(i, "a", 100, 100) for i in range(5)])
    _, take = s._take_batch()
    assert len(take) == 2 and s.in_flight_bytes == 2 * one          # the budget admits two
    _, take = s._take_batch()
    assert take == [] and len(s.pending) == 3                       # nothing fits beside them
    s.in_flight_bytes = 0                                           # the batch completed
    _, take = s._take_batch()
    assert len(take) == 2
    # a request larger than the whole budget still runs, alone, once nothing is in flight
    s = bare_server(budget=one // 2, max_rays=1 << 30)
    s.pending.extend([req(0, "a", 100, 100), req(1, "a", 100, 100)])
    _, take = s._take_batch()
    assert [r.rid for r in take] == [0]
    _, take = s._take_batch()
    assert take == []


def test_poisson_stream_is_seeded_and_has_the_requested_rate():
    names = ["g0", "g1", "g2", "g3"]
    a = SV.poisson_stream(4000, 200.0, seed=7, grids=names, resolutions=SV.RES_MIX)
    b = SV.poisson_stream(4000, 200.0, seed=7, grids=names, resolutions=SV.RES_MIX)
    c = SV.poisson_stream(4000, 200.0, seed=8, grids=names, resolutions=SV.RES_MIX)
    ta = np.array([t for t, _ in a])
    assert np.array_equal(ta, [t for t, _ in b])
    assert not np.array_equal(ta, [t for t, _ in c])
    assert np.all(np.diff(ta) > 0)
    gaps = np.diff(np.concatenate([[0.0], ta]))
    assert abs(gaps.mean() - 1 / 200.0) < 4 * (1 / 200.0) / np.sqrt(len(gaps))   # exponential mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1                            # CV of an exponential
    counts = collections.Counter(r.grid for _, r in a)
    assert set(counts) == set(names) and min(counts.values()) > 900
    res = collections.Counter((r.W, r.H) for _, r in a)
    assert set(res) == set(SV.RES_MIX) and min(res.values()) > 900
    assert [r.rid for _, r in a] == list(range(4000))
    assert all(r.cam.shape == (16,) for _, r in a[:10])
