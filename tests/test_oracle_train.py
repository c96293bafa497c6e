"""Pins of the oracle's NeuS-style training loss and its reverse-mode gradient (CPU only).

Closed forms used (Sec. 3.2.2 loss; NeuS discrete opacity; Sec. 3.3 finite differences):
  * transmittance telescopes: where d decreases along the whole ray, 1 - alpha_i = Phi_{i+1}/Phi_i,
    so T_final = Phi(s d_last) / Phi(s d_first) and a constant colour c renders C = c (1 - T_final);
  * where d increases along the ray every alpha is clamped to 0 and C = 0;
  * the central difference of a linear SDF is exact, so the eikonal term of a unit plane is 0 and
    of a plane with |grad| = 2 is exactly 1;
  * importance samples invert the CDF of the coarse NeuS weights; for a plane crossed head-on they
    follow the logistic distribution of scale 1/s_up centred on the crossing;
  * the reverse-mode gradient matches central finite differences (h = 1e-4, FP64) of the loss, and
    two of its entries have closed forms (a colour bias and the SDF output bias on a plane).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2206_10885_gb300 import synth as S
from tests import gridkit as K

pytestmark = pytest.mark.filterwarnings("ignore")


def small_desc(N=2, hidden=2, occ=0):
    return S.GridDesc(N=N, sdf_hidden=hidden, sdf_width=32, col_hidden=1, col_width=32, occ_res=occ)


def phi(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, dtype=np.float64)))


def const_colour(desc, w, rgb_logit):
    """Colour MLP with zero weights and output bias rgb_logit: colour = sigmoid(rgb_logit) everywhere."""
    return K.set_colour_linear(desc, w, [0], [[0.0], [0.0], [0.0]], rgb_logit)


def head_on_rays(B, seed, z0=2.5):
    """Rays straight down -z from random (x, y) in the box's footprint."""
    rng = np.random.default_rng(seed)
    o = np.concatenate([rng.uniform(-0.9, 0.9, (B, 2)), np.full((B, 1), z0)], 1)
    w = np.tile([0.0, 0.0, -1.0], (B, 1))
    return o, w


def strat_t(tn, tf, Ns, u):
    return tn + (np.arange(Ns) + u) / Ns * (tf - tn)


def test_transmittance_telescopes_on_a_plane():
    desc = small_desc()
    a, b = np.array([0.0, 0.0, 1.0]), -0.1
    logit = [0.3, -0.7, 1.1]
    w = const_colour(desc, K.plane_grid(desc, a, b), logit)
    B, Ns, Ni, s = 5, 16, 8, 20.0
    o, dirs = head_on_rays(B, 1)
    rng = np.random.default_rng(2)
    us, ui = rng.uniform(size=(B, Ns)), np.sort(rng.uniform(size=(B, Ni)), 1)
    target = np.zeros((B, 3))
    loss, parts, t = oracle.train_loss(desc, w, s, 64.0, o, dirs, target, us, ui, np.zeros((0, 3)), 0.1, 1e-2,
                                       want_t=True)
    # slab [1.5, 3.5] along -z from z = 2.5; d(t) = (2.5 - t) - 0.1
    assert np.all(np.diff(t, axis=1) >= 0) and t.min() >= 1.5 and t.max() <= 3.5
    b32 = float(np.float32(b))  # the weights hold b in FP32
    d_first, d_last = 2.5 - t[:, 0] + b32, 2.5 - t[:, -1] + b32
    Tf = phi(s * d_last) / phi(s * d_first)
    want = np.mean(np.sum(K.sigmoid(np.float32(logit))[None, :] * (1.0 - Tf)[:, None], 1))
    assert parts[1] == pytest.approx(0.0, abs=1e-20)
    assert parts[0] == pytest.approx(want, rel=1e-12)
    assert loss == pytest.approx(want, rel=1e-12)


def test_receding_surface_renders_black():
    desc = small_desc()
    w = const_colour(desc, K.plane_grid(desc, [0.0, 0.0, -1.0], 0.1), [0.5, 0.5, 0.5])
    B, Ns, Ni = 4, 16, 8
    o, dirs = head_on_rays(B, 3)
    rng = np.random.default_rng(4)
    loss, parts, _ = oracle.train_loss(desc, w, 20.0, 64.0, o, dirs, np.zeros((B, 3)), rng.uniform(size=(B, Ns)),
                                       np.sort(rng.uniform(size=(B, Ni)), 1), np.zeros((0, 3)), 0.1, 1e-2)
    assert parts[0] == 0.0
    # a target of 1 costs exactly 3 per ray
    loss1, parts1, _ = oracle.train_loss(desc, w, 20.0, 64.0, o, dirs, np.ones((B, 3)), rng.uniform(size=(B, Ns)),
                                         np.sort(rng.uniform(size=(B, Ni)), 1), np.zeros((0, 3)), 0.1, 1e-2)
    assert parts1[0] == pytest.approx(3.0, rel=1e-15)


def test_missed_box_and_target_only():
    desc = small_desc()
    w = const_colour(desc, K.plane_grid(desc, [0.0, 0.0, 1.0], -0.1), [2.0, 2.0, 2.0])
    o = np.array([[3.0, 3.0, 3.0]])
    dirs = np.array([[1.0, 0.0, 0.0]])
    tgt = np.array([[0.25, 0.5, 0.125]])
    _, parts, t = oracle.train_loss(desc, w, 20.0, 64.0, o, dirs, tgt, np.full((1, 4), 0.5), np.full((1, 2), 0.5),
                                    np.zeros((0, 3)), 0.1, 1e-2, want_t=True)
    assert parts[0] == pytest.approx(0.875, rel=1e-15)
    assert np.all(t == 0)


@pytest.mark.parametrize("scale,want", [(1.0, 0.0), (2.0, 1.0), (0.5, 0.25)])
def test_eikonal_of_planes(scale, want):
    desc = small_desc(N=4)
    a = scale * np.array([0.6, 0.0, 0.8])
    w = K.plane_grid(desc, a, 0.05)
    P = S.uniform(S.stream_key(5, 1), 3 * 64).reshape(64, 3) * 1.9 - 0.95
    _, parts, _ = oracle.train_loss(desc, w, 20.0, 64.0, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3)),
                                    np.zeros((0, 4)), np.zeros((0, 2)), P, 0.1, 1e-2)
    # a is rounded to FP32 in the weights
    an = np.linalg.norm(a.astype(np.float32).astype(np.float64))
    assert parts[1] == pytest.approx((an - 1.0) ** 2, abs=1e-12)
    assert parts[1] == pytest.approx(want, abs=1e-6)


def test_eikonal_seam_difference():
    """FD across a cell seam sees the jump: per-cell offsets b_c make |g| large there."""
    desc = small_desc(N=2)
    cell_b = np.array([0.0, 0.02, 0.0, 0.02, 0.0, 0.02, 0.0, 0.02])  # jump of 0.02 across x = 0
    w = K.plane_grid(desc, [0.0, 0.0, 1.0], 0.0, cell_b=cell_b)
    h = 1e-2
    P = np.array([[0.004, 0.3, 0.2], [-0.5, 0.3, 0.2]])
    _, parts, _ = oracle.train_loss(desc, w, 20.0, 64.0, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3)),
                                    np.zeros((0, 4)), np.zeros((0, 2)), P, 0.1, h)
    gx = 0.02 / (2 * h)  # x +- h straddles the seam at the first point only
    want = ((math.sqrt(gx * gx + 1.0) - 1.0) ** 2 + 0.0) / 2
    assert parts[1] == pytest.approx(want, rel=1e-6)


def test_importance_samples_follow_logistic():
    desc = small_desc()
    w = K.plane_grid(desc, [0.0, 0.0, 1.0], -0.1)
    Ns, Ni, s_up = 1024, 99, 64.0
    o = np.array([[0.05, 0.05, 2.5]])
    dirs = np.array([[0.0, 0.0, -1.0]])
    q = (np.arange(Ni) + 1.0) / (Ni + 1.0)
    _, _, t = oracle.train_loss(desc, w, 20.0, s_up, o, dirs, np.zeros((1, 3)), np.full((1, Ns), 0.5), q[None, :],
                                np.zeros((0, 3)), 0.1, 1e-2, want_t=True)
    ts = t[0]
    strat = strat_t(1.5, 3.5, Ns, 0.5)
    imp = np.array([x for x in ts if np.min(np.abs(strat - x)) > 1e-12])
    assert imp.size == Ni and np.all(np.diff(ts) >= 0)
    # continuous limit: coarse weight mass up to t is 1 - T(t) = 1 - Phi(s_up d(t)) / Phi(s_up d(t_0)), plus the
    # 1e-5 floor on each of the Ns - 1 intervals spread evenly over [t_0, t_{Ns-1}]
    tstar = 2.5 + float(np.float32(-0.1))
    t0, t1 = strat[0], strat[-1]

    def cdf(t):
        mass = 1.0 - phi(s_up * (tstar - t)) / phi(s_up * (tstar - t0))
        pad = 1e-5 * (Ns - 1) * (t - t0) / (t1 - t0)
        tot = 1.0 - phi(s_up * (tstar - t1)) / phi(s_up * (tstar - t0)) + 1e-5 * (Ns - 1)
        return (mass + pad) / tot

    lo, hi = np.full(Ni, t0), np.full(Ni, t1)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        below = cdf(mid) < q
        lo, hi = np.where(below, mid, lo), np.where(below, hi, mid)
    want = 0.5 * (lo + hi)
    assert np.max(np.abs(imp - want)) < 1e-3
    # and the bulk sits on the logistic quantiles of scale 1/s_up
    logistic = tstar + np.log(q / (1.0 - q)) / s_up
    core = (q > 0.2) & (q < 0.8)
    assert np.max(np.abs(imp[core] - logistic[core])) < 2e-3


def test_importance_at_cdf_knots_hits_sample_positions():
    """A uniform weight (d constant -> alpha 0, weights all 1e-5) puts u = k/(Ns-1) on the k-th sample."""
    desc = small_desc()
    w = K.plane_grid(desc, [0.0, 0.0, 0.0], 0.3)
    Ns = 9
    o = np.array([[0.05, 0.05, 2.5]])
    dirs = np.array([[0.0, 0.0, -1.0]])
    u = np.array([[0.125, 0.375, 0.625, 0.875]])  # k/8 for k = 1, 3, 5, 7
    _, _, t = oracle.train_loss(desc, w, 20.0, 64.0, o, dirs, np.zeros((1, 3)), np.full((1, Ns), 0.5), u,
                                np.zeros((0, 3)), 0.1, 1e-2, want_t=True)
    strat = strat_t(1.5, 3.5, Ns, 0.5)
    for k in (1, 3, 5, 7):
        assert np.sum(np.abs(t[0] - strat[k]) < 1e-12) == 2  # the stratified sample and its importance twin


# ------------------------------------------------------------------------------------ gradient

def grad_problem(seed, B=6, Ns=8, Ni=4, M=5):
    desc = small_desc(N=2, hidden=2)
    base = S.sal_sphere_grid(desc, seed=seed).reshape(desc.n_cells, desc.p_cell)
    rnd = K.random_grid(desc, seed + 7, scale=0.3).reshape(desc.n_cells, desc.p_cell)
    off = S.layer_offsets(desc)
    ns = len(desc.sdf_layers())
    base[:, off[ns][0]:] = rnd[:, off[ns][0]:]  # live colour MLP
    w = base.reshape(-1).astype(np.float32)
    cams = S.orbit_cameras(2, 8, 8, seed=seed)
    rng = np.random.default_rng(seed)
    pix = rng.integers(0, 64, size=B)
    cam = rng.integers(0, 2, size=B)
    o = np.zeros((B, 3))
    dirs = np.zeros((B, 3))
    for r in range(B):
        o[r], dirs[r] = oracle.ray(cams[cam[r]], pix[r] // 8, pix[r] % 8)
    tgt = rng.uniform(0.2, 0.8, size=(B, 3))
    us = rng.uniform(size=(B, Ns))
    ui = np.sort(rng.uniform(size=(B, Ni)), 1)
    P = rng.uniform(-0.95, 0.95, size=(M, 3))
    return desc, w, o, dirs, tgt, us, ui, P


def fd_entries(desc, w, args, t_fixed, idx, h=1e-4):
    """Central differences of the oracle loss in the FP32 weights (actual step from FP32 rounding)."""
    out = []
    for j in idx:
        wp, wm = w.copy(), w.copy()
        wp[j] = np.float32(w[j] + h)
        wm[j] = np.float32(w[j] - h)
        lp, _, _ = oracle.train_loss(desc, wp, *args, t_fixed=t_fixed)
        lm, _, _ = oracle.train_loss(desc, wm, *args, t_fixed=t_fixed)
        out.append((lp - lm) / (float(wp[j]) - float(wm[j])))
    return np.array(out)


def test_gradient_matches_central_differences():
    desc, w, o, dirs, tgt, us, ui, P = grad_problem(11)
    s, s_up, lam, h = 20.0, 64.0, 0.1, 1e-2
    args = (s, s_up, o, dirs, tgt, us, ui, P, lam, h)
    loss, parts, t = oracle.train_loss(desc, w, *args, want_t=True)
    loss_g, _, g = oracle.train_grad(desc, w, *args)
    assert loss_g == loss
    # every parameter group of every cell: sample entries where the gradient is not tiny
    rng = np.random.default_rng(0)
    live = np.flatnonzero(np.abs(g) > 1e-6 * np.abs(g).max())
    idx = rng.choice(live, size=min(160, live.size), replace=False)
    fd = fd_entries(desc, w, args, t, idx)
    err = np.abs(fd - g[idx])
    ok = err <= 1e-7 + 2e-4 * np.abs(g[idx])
    assert ok.mean() >= 0.97, (np.sort(err / (np.abs(g[idx]) + 1e-12))[-10:])
    assert np.median(err / np.abs(g[idx])) < 1e-6
    # entries no sample touches have zero gradient (t fixed; cells without samples)
    assert np.all(np.isfinite(g))


def test_gradient_closed_forms_on_a_plane():
    """N = 1: one cell.  Constant colour c = sigmoid(b_c), target 0, rays head-on, d decreasing.

    dL/db_c[q] = mean_r (1 - T_r) c_q (1 - c_q);  dL/d(d-row bias) = -mean_r sum_q c_q s (Phi_l/Phi_0)(Phi_0 - Phi_l).
    """
    desc = small_desc(N=1)
    logit = np.array([0.3, -0.7, 1.1])
    w = const_colour(desc, K.plane_grid(desc, [0.0, 0.0, 1.0], -0.1), logit)
    B, Ns, Ni, s = 5, 16, 8, 20.0
    o, dirs = head_on_rays(B, 1)
    rng = np.random.default_rng(2)
    us, ui = rng.uniform(size=(B, Ns)), np.sort(rng.uniform(size=(B, Ni)), 1)
    P = np.zeros((0, 3))
    _, _, t = oracle.train_loss(desc, w, s, 64.0, o, dirs, np.zeros((B, 3)), us, ui, P, 0.1, 1e-2, want_t=True)
    _, _, g = oracle.train_grad(desc, w, s, 64.0, o, dirs, np.zeros((B, 3)), us, ui, P, 0.1, 1e-2)
    c = K.sigmoid(logit.astype(np.float32))
    b32 = float(np.float32(-0.1))
    p0, pl = phi(s * (2.5 - t[:, 0] + b32)), phi(s * (2.5 - t[:, -1] + b32))
    T = pl / p0
    off = S.layer_offsets(desc)
    ns = len(desc.sdf_layers())
    b_col = off[ns + 1][1]
    np.testing.assert_allclose(g[b_col:b_col + 3], np.mean(1.0 - T) * c * (1 - c), rtol=1e-10)
    b_d = off[ns - 1][1]
    want = -np.mean(np.sum(c) * s * T * (p0 - pl))
    assert g[b_d] == pytest.approx(want, rel=1e-9)


def test_gradient_eikonal_only_closed_form():
    """Plane with |grad d| = 2 and no rays: L = lam (2 - 1)^2, and a shift of d (its output bias)
    cancels in every central difference, so that bias gets exactly no gradient."""
    desc = small_desc(N=1)
    w = K.plane_grid(desc, [0.0, 0.0, 2.0], 0.0)
    P = np.array([[0.1, 0.2, 0.3], [-0.4, 0.5, -0.6]])
    args = (20.0, 64.0, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 4)), np.zeros((0, 2)), P,
            0.1, 1e-2)
    loss, parts, g = oracle.train_grad(desc, w, *args)
    assert loss == pytest.approx(0.1, rel=1e-12)
    off = S.layer_offsets(desc)
    ns = len(desc.sdf_layers())
    assert g[off[ns - 1][1]] == 0.0
    # the colour MLP is not used by the eikonal term
    assert np.all(g[off[ns][0]:] == 0.0)
