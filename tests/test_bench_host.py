"""Host arithmetic of the bench (CPU only): the algorithmic multiply-add counts the roofline divides
by, checked against the layer shapes written out by hand, and the rule that takes the roofline's
traffic figure from a committed capture only while the kernel's sources are unchanged."""
from __future__ import annotations

import os
import sys

from paper_2206_10885_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_render_mac_counts():
    import bench
    # width 32, 3 hidden layers, L = 4: 27 -> 32 -> 32 -> 32 -> d
    assert bench.mac_counts(S.config_desc("c2")) == (27 * 32 + 2 * 32 * 32 + 32,
                                                     # full forward [d, z] + backward to the input
                                                     # + colour 33 -> 32 -> 3
                                                     (27 * 32 + 2 * 32 * 32 + 32 * 16) + (2 * 32 * 32 + 27 * 32)
                                                     + (33 * 32 + 32 * 3))
    assert bench.mac_counts(S.config_desc("c2")) == (2944, 7488)
    assert bench.mac_counts(S.config_desc("c3l")) == (9984, 23168)
    assert bench.mac_counts(S.config_desc("c1"))[0] == 27 * 32 + 32 * 32 + 32


def test_training_mac_counts():
    import bench
    m = bench.train_macs(S.config_desc(S.TRAIN_WORKLOAD["grid"]))
    assert m == {"fwd_d": 2944, "fwd_full": 4576, "bwd_d": 5024, "bwd_full": 7808}


def test_profile_traffic_is_used_only_while_the_kernel_sources_match(tmp_path, monkeypatch):
    """The roofline's traffic figure comes from a committed capture summary only while the sources of
    its kernel hash to the summary's hash; an edited kernel makes it None (stale counters)."""
    import bench
    csrc = tmp_path / "paper_2206_10885_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in bench.KERNEL_SOURCES["trace_tc_kernel"]:
        (csrc / fn).write_text("// %s\n" % fn)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("trace_tc_kernel_bf16_c3l")
    (tmp_path / "profiles" / "x.md").write_text(
        "kernel_tag: trace_tc_kernel_bf16_c3l\nkernel_source_sha1: %s\ndram_bytes_per_full_launch: 4.12e8\n" % h)
    assert bench.profile_traffic("trace_tc_kernel_bf16_c3l") == 4.12e8
    assert bench.profile_traffic("trace_tc_kernel_bf16_c3s") is None      # another workload's tag
    (csrc / "kns_tc.cu").write_text("// edited\n")
    assert bench.profile_traffic("trace_tc_kernel_bf16_c3l") is None      # the kernel changed since

