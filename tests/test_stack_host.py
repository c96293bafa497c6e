"""Host side of grid stacks (CPU only): the Python binding's marshalling of a stack upload and of the
grid index of each view, with the C calls replaced by recorders (no device is touched)."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import paper_2206_10885_gb300 as kns
from paper_2206_10885_gb300 import _capi as capi
from paper_2206_10885_gb300 import synth as S


class _Ctx:
    handle, device = 1234, 0


def test_load_stack_passes_the_grids_back_to_back(monkeypatch):
    desc = S.config_desc("c1")
    ws = [np.full(10, k, dtype=np.float32) for k in range(3)]
    occ = [np.full(4, 7 + k, dtype=np.uint64) for k in range(3)]
    seen = {}

    def fake(ctx, d, n, wptr, nf, optr):
        seen["args"] = (ctx, n, nf)
        seen["w"] = np.ctypeslib.as_array((C.c_float * nf).from_address(wptr)).copy()
        seen["occ"] = np.ctypeslib.as_array((C.c_uint64 * 12).from_address(optr)).copy() if optr else None
        return 99

    monkeypatch.setattr(capi, "kns_load_grid_stack", fake)
    g = kns.Grid.load_stack(_Ctx(), desc, ws, occ)
    assert g.handle == 99
    assert seen["args"] == (1234, 3, 30)
    assert np.array_equal(seen["w"], np.repeat(np.arange(3, dtype=np.float32), 10))  # grid k's weights k-th
    assert np.array_equal(seen["occ"], np.repeat(np.arange(7, 10, dtype=np.uint64), 4))
    g.handle = None
    kns.Grid.load_stack(_Ctx(), desc, ws)
    assert seen["occ"] is None  # no masks given: each grid's is built on the device


def test_render_views_sets_each_views_grid(monkeypatch):
    torch = pytest.importorskip("torch")
    seen = {}

    def fake(ctx, grid, arr, max_steps, eps, opts, stream):
        seen["views"] = [(arr[i].W, arr[i].H, arr[i].grid, arr[i].reserved) for i in range(len(arr))]
        seen["cam0"] = [arr[0].cam.c2w[k] for k in range(3)]

    monkeypatch.setattr(capi, "kns_render_views", fake)
    monkeypatch.setattr(kns, "_stream_ptr", lambda s: 0)
    cam = np.arange(16, dtype=np.float32)
    reqs = [(cam, 4, 3), (cam, 2, 2, 1), (cam, 1, 5, 2)]
    outs = [kns.alloc_frame(W * H, "cpu") for _, W, H, *rest in reqs]
    kns.render_views(_Ctx(), type("G", (), {"handle": 5})(), reqs, 64, 1e-4, outs=outs)
    assert seen["views"] == [(4, 3, 0, 0), (2, 2, 1, 0), (1, 5, 2, 0)]  # absent index: grid 0
    assert seen["cam0"] == [0.0, 1.0, 2.0]


def test_view_struct_layout_keeps_its_outputs_in_place():
    # the grid index follows the output pointers, so a caller's view layout up to them is unchanged
    assert capi.kns_view.out.offset == 16 * 4 + 2 * 4
    assert capi.kns_view.grid.offset == capi.kns_view.out.offset + C.sizeof(capi.kns_frame)
