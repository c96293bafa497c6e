"""C ABI checks that need no GPU: the library loads, exports every declared entry point,
the ctypes structures match the header's layout, and host-side argument checks return the
documented status codes without touching a device."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2206_10885_gb300 import _capi as capi
from paper_2206_10885_gb300 import build as kbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return capi.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(kns_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "kns_render" in names and "kns_sdf" in names and "kns_load_grid" in names
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", capi.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (kns_\w+)", out))
    assert exported == set(names)
    # nothing but the C ABI is exported (the CUDA runtime inside stays private)
    assert all(line.split()[-1].startswith("kns_") for line in out.splitlines() if " T " in line)


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "kns.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(kns_grid_desc), sizeof(kns_camera), sizeof(kns_frame), sizeof(kns_render_opts));
  printf("%zu %zu %zu\\n", offsetof(kns_grid_desc, softplus_beta), offsetof(kns_grid_desc, bbox_max),
         offsetof(kns_camera, cy));
  printf("%zu %zu %zu\\n", offsetof(kns_frame, hit), offsetof(kns_render_opts, refine_steps),
         offsetof(kns_render_opts, block_tiles));
  printf("%zu %zu %zu %zu\\n", sizeof(kns_train_batch), offsetof(kns_train_batch, n_eik),
         offsetof(kns_train_batch, s), offsetof(kns_train_batch, timing));
  printf("%zu %zu\\n", sizeof(kns_train_stats), offsetof(kns_train_stats, ms_fd_backward));
  printf("%zu %zu %zu\\n", sizeof(kns_pt_opts), offsetof(kns_pt_opts, seed), offsetof(kns_pt_opts, zenith));
  printf("%zu %zu %zu\\n", sizeof(kns_render_stats), offsetof(kns_render_stats, ms_eval_fp32),
         offsetof(kns_render_stats, refined));
  printf("%zu %zu\\n", sizeof(kns_round_info), offsetof(kns_round_info, tiles));
  printf("%zu %zu\\n", sizeof(kns_peaks), offsetof(kns_peaks, sm_clock_khz));
  printf("%zu %zu %zu\\n", sizeof(kns_view), offsetof(kns_view, out), offsetof(kns_view, grid));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [C.sizeof(capi.kns_grid_desc), C.sizeof(capi.kns_camera), C.sizeof(capi.kns_frame),
            C.sizeof(capi.kns_render_opts), capi.kns_grid_desc.softplus_beta.offset,
            capi.kns_grid_desc.bbox_max.offset, capi.kns_camera.cy.offset, capi.kns_frame.hit.offset,
            capi.kns_render_opts.refine_steps.offset, capi.kns_render_opts.block_tiles.offset,
            C.sizeof(capi.kns_train_batch),
            capi.kns_train_batch.n_eik.offset, capi.kns_train_batch.s.offset, capi.kns_train_batch.timing.offset,
            C.sizeof(capi.kns_train_stats), capi.kns_train_stats.ms_fd_backward.offset,
            C.sizeof(capi.kns_pt_opts), capi.kns_pt_opts.seed.offset, capi.kns_pt_opts.zenith.offset,
            C.sizeof(capi.kns_render_stats), capi.kns_render_stats.ms_eval_fp32.offset,
            capi.kns_render_stats.refined.offset,
            C.sizeof(capi.kns_round_info), capi.kns_round_info.tiles.offset,
            C.sizeof(capi.kns_peaks), capi.kns_peaks.sm_clock_khz.offset,
            C.sizeof(capi.kns_view), capi.kns_view.out.offset, capi.kns_view.grid.offset]
    assert vals == want


def test_null_context_is_rejected_on_the_host(lib):
    assert lib.kns_render(None, None, None, 1, 1, 1, 1, 1e-4, None, None, None) == capi.KNS_ERR_INVALID_ARG
    assert lib.kns_sdf(None, None, None, 0, None, None, None, None) == capi.KNS_ERR_INVALID_ARG
    assert lib.kns_sync(None, None, 0) == capi.KNS_ERR_INVALID_ARG
    h = C.c_void_p()
    assert lib.kns_load_grid(None, None, None, 0, None, C.byref(h)) == capi.KNS_ERR_INVALID_ARG
    assert lib.kns_create(0, None) == capi.KNS_ERR_INVALID_ARG
    assert "NULL" in capi.kns_last_error(None)
    lib.kns_destroy(None)
    lib.kns_free_grid(None)
    # every entry point that takes a context refuses NULL before touching the device
    bad = capi.KNS_ERR_INVALID_ARG
    assert lib.kns_render_noalloc(None, None, None, 1, 1, 1, 1, 1e-4, None, None) == bad
    assert lib.kns_render_views(None, None, None, 1, 1, 1e-4, None, None) == bad
    assert lib.kns_get_render_stats(None, None) == bad
    assert lib.kns_get_round_trace(None, None, 0, None) == bad
    assert lib.kns_measure_peaks(None, None, None) == bad
    assert lib.kns_trace_rays(None, None, None, None, 1, 1, 1e-4, None, None, None) == bad
    assert lib.kns_path_trace(None, None, None, 1, 1, 1, None, 1, 1e-4, None, None, None) == bad
    assert lib.kns_train_forward(None, None, None, None, None, None, None, None, None) == bad
    assert lib.kns_train_backward(None, 1, None, None, None) == bad
    assert lib.kns_train_step(None, None, None, None, None, None, None) == bad
    assert lib.kns_train_get_stats(None, None) == bad
    assert lib.kns_copy_occupancy(None, None, None, 0) == bad
    assert lib.kns_grid_get_desc(None, None) == bad
    assert lib.kns_load_grid_file(None, None, C.byref(h)) == bad
    assert lib.kns_load_grid_stack(None, None, 2, None, 0, None, C.byref(h)) == bad
    n = C.c_int32(0)
    assert lib.kns_grid_stack_size(None, C.byref(n)) == bad


def test_create_without_a_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(capi.KnsError) as e:
        capi.kns_create(0)
    assert e.value.status in (capi.KNS_ERR_CUDA, capi.KNS_ERR_INVALID_ARG)


def test_a_missing_library_raises_instead_of_falling_back(monkeypatch, tmp_path):
    """The product path has no CPU fallback: without libkns.so every call fails loudly."""
    monkeypatch.setattr(capi, "_lib", None)
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "libkns.so"))
    with pytest.raises(ImportError, match="not built"):
        capi.lib()
    with pytest.raises(ImportError):
        capi.kns_create(0)
