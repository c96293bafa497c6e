"""Comparison helpers for CUDA-vs-oracle parity tests (test infrastructure).

Tolerances (FP32 path):
  - hit, cell and step count: identical on every decision-robust ray, and identical on
    >= 99.9% of all rays.  A ray is decision-robust when the oracle's conditioning-aware
    margins (computed with a per-step FP32 error model of DELTA_STEP) show no threshold test
    within DELTA_D of |d| = eps and none within DELTA_X of a cell or voxel face, of the box
    interval's ends, or of a DDA axis tie;
  - on robust rays both sides hit: depth within 1e-4 scene units, RGB within 1e-5 per channel,
    normal within 1e-4 per component;
  - the robust fraction is reported, and held to a per-case floor where the test gives one (on the
    SAL grids, whose SDF is not 1-Lipschitz, 65-97 % of rays are robust);
  - on every other hit where both sides took the same decisions (same hit, cell and step count), the
    same depth, RGB and normal bounds: the only rays left unchecked are those whose decisions differ,
    at most 1 - min_agree of them.
"""
import numpy as np

import oracle as O

DELTA_STEP = 2e-6  # bound on |d_fp32 - d_fp64| of one SDF evaluation (measured by the sdf tests)
DELTA_D = 2e-6
DELTA_X = 1e-5
TOL_DEPTH = 1e-4
TOL_RGB = 1e-5
TOL_NORMAL = 1e-4


def to_np(t):
    return {k: v.detach().cpu().numpy() for k, v in t.items()}


def compare_render(gpu: dict, ora: dict, min_agree: float = 0.999, tol_depth=TOL_DEPTH, tol_rgb=TOL_RGB,
                   tol_normal=TOL_NORMAL, delta_d=DELTA_D, delta_x=DELTA_X, label="", min_robust: float = None,
                   report: list = None):
    """gpu: per-ray numpy arrays (same rays as ora).  Returns a summary dict; asserts the gates.

    Gates: (1) identical hit, cell and step count on every decision-robust ray, and on >= min_agree of
    all rays; (2) on robust hits, depth / RGB / normal within TOL_*; (3) the robust fraction is reported
    and, given min_robust, held to it; (4) on every other hit where both sides took the same decisions
    (same hit, cell and steps -- the near-threshold rays the robust set leaves out), depth, RGB and normal
    within the same tol_*, so the only rays left unchecked are those whose decisions differ."""
    n = ora["hit"].shape[0]
    g_hit = gpu["hit"].astype(bool)
    o_hit = ora["hit"].astype(bool)
    robust = O.robust_mask(ora["margins"], delta_d, delta_x)
    same_dec = (g_hit == o_hit) & (gpu["cell"] == ora["cell"]) & (gpu["steps"] == ora["steps"])
    bad_robust = np.where(robust & ~same_dec)[0]
    assert bad_robust.size == 0, (label, "robust rays disagree", bad_robust[:10], gpu["steps"][bad_robust[:5]],
                                  ora["steps"][bad_robust[:5]], ora["margins"][bad_robust[:5]])
    agree = float(np.mean(same_dec))
    assert agree >= min_agree, (label, "decision agreement", agree)
    both = g_hit & o_hit & same_dec & robust
    dd = np.abs(gpu["depth"][both].astype(np.float64) - ora["depth"][both])
    dr = np.abs(gpu["rgb"][both].astype(np.float64) - ora["rgb"][both])
    dn = np.abs(gpu["normal"][both].astype(np.float64) - ora["normal"][both])
    # hits the robust set leaves out, where both sides still took the same decisions
    rest = g_hit & o_hit & same_dec & ~robust
    rd = np.abs(gpu["depth"][rest].astype(np.float64) - ora["depth"][rest])
    rr = np.abs(gpu["rgb"][rest].astype(np.float64) - ora["rgb"][rest]).max(axis=1) if rest.any() else np.zeros(0)
    rn = np.abs(gpu["normal"][rest].astype(np.float64) - ora["normal"][rest]).max(axis=1) if rest.any() else np.zeros(0)
    rest_ok = (rd <= tol_depth) & (rr <= tol_rgb) & (rn <= tol_normal)
    summary = dict(n=n, hits=int(o_hit.sum()), robust=float(robust.mean()), robust_rays=int(robust.sum()),
                   robust_hits=int(both.sum()), agree=agree,
                   max_depth_err=float(dd.max()) if dd.size else 0.0,
                   max_rgb_err=float(dr.max()) if dr.size else 0.0,
                   max_normal_err=float(dn.max()) if dn.size else 0.0,
                   other_same_decision_hits=int(rest.sum()),
                   other_within_tol=float(rest_ok.mean()) if rest.any() else 1.0,
                   other_max_depth_err=float(rd.max()) if rd.size else 0.0,
                   other_max_rgb_err=float(rr.max()) if rr.size else 0.0,
                   other_max_normal_err=float(rn.max()) if rn.size else 0.0)
    print("parity", label, summary)
    if report is not None:
        report.append(dict(summary, label=label))
    if dd.size:
        assert dd.max() <= tol_depth, (label, summary)
        assert dr.max() <= tol_rgb, (label, summary)
        assert dn.max() <= tol_normal, (label, summary)
    if rest.any():
        assert rest_ok.all(), (label, "same-decision hits outside the robust set", summary)
    if min_robust is not None:
        assert summary["robust"] >= min_robust, (label, "robust fraction", summary)
    misses = ~g_hit
    assert np.all(np.isinf(gpu["depth"][misses])) and np.all(gpu["rgb"][misses] == 0)
    assert np.all(gpu["cell"][misses] == -1)
    return summary
