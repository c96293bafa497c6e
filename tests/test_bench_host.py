"""Host arithmetic of the bench (CPU only): the algorithmic multiply-add counts the roofline divides
by, checked against the layer shapes written out by hand."""
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
