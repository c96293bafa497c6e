"""Host logic of the schedule autotuner (CPU only): the candidate set it times."""
from __future__ import annotations

import itertools

from paper_2206_10885_gb300 import autotune as A


def test_candidates_cover_the_space_without_duplicates():
    cands = list(A.candidates())
    keys = set(A.SPACE)
    assert all(set(c) == keys for c in cands)
    assert len({tuple(sorted(c.items())) for c in cands}) == len(cands)
    for c in cands:
        for k, v in c.items():
            assert v in A.SPACE[k] or A.WARP_ONLY.get(k) == v


def test_block_tiles_fix_only_the_warp_tile_knobs():
    cands = list(A.candidates())
    block = [c for c in cands if c["block_tiles"] != 2]
    warp = [c for c in cands if c["block_tiles"] == 2]
    # block tiles size their own grid: one value of the warp-only knob ...
    assert {c["blocks_per_sm"] for c in block} == {A.WARP_ONLY["blocks_per_sm"]}
    # ... but take the in-tile stepping knobs like the warp tiles do
    for k in ("inner_steps", "min_active", "tail_rays", "static_tiles"):
        assert {c[k] for c in block} == set(A.SPACE[k])
        assert {c[k] for c in warp} == set(A.SPACE[k])
    assert {c["blocks_per_sm"] for c in warp} == set(A.SPACE["blocks_per_sm"])
    # every combination of the remaining knobs appears exactly once per tile kind
    free = [k for k in sorted(A.SPACE) if k not in A.WARP_ONLY and k != "block_tiles"]
    n_free = 1
    for k in free:
        n_free *= len(A.SPACE[k])
    n_block_kinds = len([b for b in A.SPACE["block_tiles"] if b != 2])
    assert len(block) == n_block_kinds * n_free
    assert len(warp) == n_free * len(A.SPACE["blocks_per_sm"])


def test_explicit_space_is_respected():
    space = {"block_tiles": (1,), "inner_steps": (1, 2), "min_active": (16,), "static_tiles": (2,),
             "blocks_per_sm": (8, 16), "tail_rays": (-1,)}
    cands = list(A.candidates(space))
    assert sorted(c["inner_steps"] for c in cands) == [1, 2]
    assert all(c["blocks_per_sm"] == 16 for c in cands)
    got = {tuple(sorted(c.items())) for c in cands}
    want = {tuple(sorted(dict(zip(sorted(space), v), blocks_per_sm=16).items()))
            for v in itertools.product(*(space[k] for k in sorted(space)))}
    assert got == want


def test_bf16_space_is_the_bf16_knobs():
    assert A.space_for(1) is A.SPACE_BF16 and A.space_for(0) is A.SPACE
    cands = list(A.candidates(A.SPACE_BF16))
    n = 1
    for v in A.SPACE_BF16.values():
        n *= len(v)
    assert len(cands) == n
    assert all(set(c) == {"tail_rays", "bf16_inner_steps", "bf16_min_active"} for c in cands)
    assert all(c["tail_rays"] > 0 and 1 <= c["bf16_inner_steps"] <= 1024 and 1 <= c["bf16_min_active"] <= 128
               for c in cands)
