"""Autotuner of the render schedule (the tuning fields of kns_render_opts).

The knobs change only how work is scheduled on the device (rounds, in-tile steps, tile hand-out,
launch width, tail).  FP32 renders are bit-identical across settings (tested); a BF16 render's
results depend on which rays reach the FP32 tail, within the BF16 accuracy gates (tested at the
defaults and across the schedule forms).  tune() times each candidate with CUDA events around kns_render, flushing L2
between repetitions, and returns the fastest setting.  Results are cached per (device, grid shape,
image shape, precision) in a JSON file next to this module (or the path in KNS_TUNE_CACHE).
"""
from __future__ import annotations

import itertools
import json
import os
import time

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(_HERE, "_tune_cache.json")

# candidate values of each knob (0 would mean the library default)
SPACE = {
    "block_tiles": (1, 2, 3, 4),
    "inner_steps": (1, 2, 4),
    "min_active": (1, 8, 32),
    "static_tiles": (1, 2),
    "blocks_per_sm": (8, 16, 32),
    "tail_rays": (-1, 131072, 262144, 524288),
}
# BF16 renders: the hand-over to the FP32 tail and the tensor-core tiles' in-tile evaluations
SPACE_BF16 = {
    "tail_rays": (8192, 16384, 24576, 32768, 65536),
    "bf16_inner_steps": (1, 2, 4, 8),
    "bf16_min_active": (4, 16, 32),
}


def space_for(precision: int):
    """The default search space of a precision (0 = FP32, 1 = BF16)."""
    return SPACE_BF16 if precision == 1 else SPACE


def _key(grid, n_cams, W, H, max_steps, precision, device_name):
    d = grid.desc
    return "|".join(str(v) for v in ("v3", device_name, d.N, d.sdf_width, d.sdf_hidden, d.pe_pos_L, d.occ_res,
                                      n_cams, W, H, max_steps, precision))


def _cache_path():
    return os.environ.get("KNS_TUNE_CACHE", DEFAULT_CACHE)


def load_cached(key):
    try:
        with open(_cache_path()) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def _store(key, value):
    path = _cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[key] = value
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


# knobs that only the 16-sample warp tiles read (block tiles size their own grid)
WARP_ONLY = {"blocks_per_sm": 16}


def candidates(space=None):
    space = space or SPACE
    keys = sorted(space)
    seen = set()
    for vals in itertools.product(*(space[k] for k in keys)):
        cand = dict(zip(keys, vals))
        if cand.get("block_tiles") in (1, 3, 4):
            cand.update({k: v for k, v in WARP_ONLY.items() if k in cand})
        key = tuple(sorted(cand.items()))
        if key not in seen:
            seen.add(key)
            yield cand


def time_setting(kns, ctx, grid, cams, W, H, max_steps, eps, precision, tuning, out, flush, reps=2):
    import torch
    stream = torch.cuda.current_stream()
    kns.render(ctx, grid, cams, W, H, max_steps, eps, precision=precision, out=out, stream=stream, tuning=tuning)
    best = float("inf")
    for k in range(reps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        kns.render(ctx, grid, cams, W, H, max_steps, eps, precision=precision, out=out, stream=stream,
                   tuning=tuning)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    ctx.sync(stream)
    return best


def tune(ctx, grid, cams, W, H, max_steps, eps, precision=0, space=None, use_cache=True, budget_s=120.0,
         verbose=False):
    """Returns (best tuning dict, best ms, list of (tuning, ms)) for this workload shape."""
    import torch

    import paper_2206_10885_gb300 as kns
    dev = torch.cuda.get_device_name(ctx.device)
    key = _key(grid, len(cams), W, H, max_steps, precision, dev)
    if use_cache:
        hit = load_cached(key)
        if hit:
            return hit["tuning"], hit["ms"], []
    out = kns.alloc_frame(len(cams) * W * H, "cuda:%d" % ctx.device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda:%d" % ctx.device)
    results = []
    t_start = time.time()
    for tuning in candidates(space or space_for(precision)):
        ms = time_setting(kns, ctx, grid, cams, W, H, max_steps, eps, precision, tuning, out, flush)
        results.append((tuning, ms))
        if verbose:
            print("tune", tuning, "%.3f ms" % ms, flush=True)
        if time.time() - t_start > budget_s:
            break
    best, best_ms = min(results, key=lambda x: x[1])
    _store(key, {"tuning": best, "ms": best_ms})
    return best, best_ms, results
