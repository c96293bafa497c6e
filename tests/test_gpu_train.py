"""Parity of the training step (kns_train_*) with the FP64 oracle: loss, sample positions, rendered
colours and the gradient of every weight; central differences (h = 1e-4, FP64) of the oracle loss;
the autograd wrapper; the full-size workload on sampled outputs and gradient properties."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2206_10885_gb300 import synth as S
from tests import gridkit as K

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_10885_gb300 as kns
    return kns


@pytest.fixture(scope="module")
def ctx(kns):
    c = kns.Context(0)
    yield c
    c.close()


def desc_of(N, H):
    return S.GridDesc(N=N, sdf_hidden=H, sdf_width=32, col_hidden=1, col_width=32, occ_res=0)


def train_weights(desc, seed):
    """SAL sphere with a live colour MLP (the trained model)."""
    return S.sal_sphere_grid(desc, seed=seed, perturb_std=1e-3)


def problem(desc, B, Ns, Ni, M, seed, n_cams=4, W=24, H=24):
    cams = S.orbit_cameras(n_cams, W, H, seed=seed + 1)
    sel, u_s, u_i, P = S.train_draws(B, Ns, Ni, M, n_cams * W * H, seed)
    o, d = S.pixel_rays(cams, W, H, sel)
    tdesc = S.GridDesc(N=desc.N, sdf_hidden=desc.sdf_hidden, sdf_width=32, col_hidden=1, col_width=32, occ_res=0)
    tw = S.sal_sphere_grid(tdesc, seed=3, perturb_std=1e-2)
    tgt = oracle.render(tdesc, tw, None, cams, W, H, 128, 1e-4, sel=sel)["rgb"].astype(np.float32)
    return dict(o=o, d=d, target=tgt, u_s=u_s, u_i=u_i, P=P)


def gpu_batch(kns, pr, s=20.0, s_up=64.0, lam=0.1, h=1e-2, t_fixed=None):
    dev = "cuda:0"
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    return kns.train.TrainBatch(f(pr["o"]), f(pr["d"]), f(pr["target"]), f(pr["u_s"]), f(pr["u_i"]), f(pr["P"]),
                                s=s, s_up=s_up, lam=lam, h=h, t_fixed=None if t_fixed is None else f(t_fixed))


def oracle_args(pr, s=20.0, s_up=64.0, lam=0.1, h=1e-2):
    d = lambda a: np.asarray(a, dtype=np.float64)
    return (s, s_up, d(pr["o"]), d(pr["d"]), d(pr["target"]), d(pr["u_s"]), d(pr["u_i"]), d(pr["P"]), lam, h)


def assert_grad_close(g_gpu, g_ref, rtol, frac=0.999, norm_tol=1e-4, what="gradient"):
    scale = np.abs(g_ref).max()
    err = np.abs(g_gpu - g_ref)
    ok = err <= rtol * np.abs(g_ref) + 1e-5 * scale
    rel_norm = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    worst = np.argsort(-err / (np.abs(g_ref) + 1e-5 * scale))[:5]
    assert ok.mean() >= frac and rel_norm <= norm_tol, (
        "%s: %.5f within tolerance, relative L2 error %.2e; worst entries %s gpu %s ref %s"
        % (what, ok.mean(), rel_norm, worst, g_gpu[worst], g_ref[worst]))


CASES = [(2, 2, 48, 16, 8, 24), (4, 3, 64, 24, 12, 40)]


@pytest.mark.parametrize("N,H,B,Ns,Ni,M", CASES)
def test_loss_samples_and_colours_match_oracle(kns, ctx, N, H, B, Ns, Ni, M):
    desc = desc_of(N, H)
    w = train_weights(desc, seed=N)
    pr = problem(desc, B, Ns, Ni, M, seed=10 + N)
    params = torch.from_numpy(w).cuda()
    loss, tok, rgb, t = kns.train.forward(ctx, desc, params, gpu_batch(kns, pr), want_rgb=True, want_t=True)
    torch.cuda.synchronize()
    l_ref, parts_ref, t_ref, rgb_ref = oracle.train_loss(desc, w, *oracle_args(pr), want_t=True, want_rgb=True)
    loss = loss.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(loss[1:], parts_ref, rtol=2e-5, atol=1e-7)
    assert loss[0] == pytest.approx(l_ref, rel=2e-5)
    # importance positions invert a CDF built from FP32 SDF values at sharpness s_up: an SDF error
    # of ~1e-6 moves a CDF knot by ~s_up 1e-6 and an importance sample by that over the local density
    t = t.cpu().numpy()
    err_t = np.abs(t - t_ref) / np.maximum(1.0, np.abs(t_ref))
    assert np.mean(err_t <= 1e-5) >= 0.9 and np.mean(err_t <= 1e-3) >= 0.99, np.percentile(err_t, [50, 90, 99, 100])
    assert np.all(np.diff(t, axis=1) >= 0)
    np.testing.assert_allclose(rgb.cpu().numpy(), rgb_ref, atol=2e-5)


@pytest.mark.parametrize("N,H,B,Ns,Ni,M", CASES)
def test_gradient_matches_oracle(kns, ctx, N, H, B, Ns, Ni, M):
    """Same sample positions on both sides (the oracle's, given as t_fixed): every weight's gradient."""
    desc = desc_of(N, H)
    w = train_weights(desc, seed=N)
    pr = problem(desc, B, Ns, Ni, M, seed=20 + N)
    args = oracle_args(pr)
    _, _, t_ref = oracle.train_loss(desc, w, *args, want_t=True)
    l_ref, parts_ref, g_ref = oracle.train_grad(desc, w, *args, t_fixed=t_ref)
    params = torch.from_numpy(w).cuda()
    loss, g = kns.train.step(ctx, desc, params, gpu_batch(kns, pr, t_fixed=t_ref))
    torch.cuda.synchronize()
    assert float(loss[0]) == pytest.approx(l_ref, rel=2e-5)
    assert_grad_close(g.cpu().numpy().astype(np.float64), g_ref, rtol=2e-3)


def test_gradient_matches_central_differences(kns, ctx):
    """dL/dw of the hand-written backward against (L(w + h e) - L(w - h e)) / 2h of the FP64 oracle."""
    desc = desc_of(2, 2)
    w = train_weights(desc, seed=5)
    pr = problem(desc, 32, 12, 6, 16, seed=33)
    args = oracle_args(pr)
    _, _, t_ref = oracle.train_loss(desc, w, *args, want_t=True)
    params = torch.from_numpy(w).cuda()
    _, g = kns.train.step(ctx, desc, params, gpu_batch(kns, pr, t_fixed=t_ref))
    g = g.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(1)
    live = np.flatnonzero(np.abs(g) > 1e-4 * np.abs(g).max())
    idx = rng.choice(live, size=min(120, live.size), replace=False)
    fd = []
    for j in idx:
        wp, wm = w.copy(), w.copy()
        wp[j] = np.float32(w[j] + 1e-4)
        wm[j] = np.float32(w[j] - 1e-4)
        lp = oracle.train_loss(desc, wp, *args, t_fixed=t_ref)[0]
        lm = oracle.train_loss(desc, wm, *args, t_fixed=t_ref)[0]
        fd.append((lp - lm) / (float(wp[j]) - float(wm[j])))
    fd = np.array(fd)
    ok = np.abs(g[idx] - fd) <= 2e-3 * np.abs(fd) + 1e-6 * np.abs(g).max()
    assert ok.mean() >= 0.97, np.sort(np.abs(g[idx] - fd) / np.abs(fd))[-8:]
    assert np.median(np.abs(g[idx] - fd) / np.abs(fd)) < 1e-4


def test_gradient_with_own_sample_placement(kns, ctx):
    """Each side places its own samples (FP32 vs FP64 CDF inversion): the gradient still agrees."""
    desc = desc_of(4, 3)
    w = train_weights(desc, seed=7)
    pr = problem(desc, 64, 24, 12, 40, seed=41)
    _, _, g_ref = oracle.train_grad(desc, w, *oracle_args(pr))
    params = torch.from_numpy(w).cuda()
    _, g = kns.train.step(ctx, desc, params, gpu_batch(kns, pr))
    assert_grad_close(g.cpu().numpy().astype(np.float64), g_ref, rtol=1e-2, frac=0.99, norm_tol=1e-2)


def test_autograd_function_and_upstream_scale(kns, ctx):
    desc = desc_of(2, 2)
    w = train_weights(desc, seed=9)
    pr = problem(desc, 40, 16, 8, 20, seed=51)
    batch = gpu_batch(kns, pr)
    p = torch.nn.Parameter(torch.from_numpy(w).cuda())
    loss, parts = kns.train.neus_loss(ctx, desc, p, batch, return_parts=True)
    (3.0 * loss).backward()
    _, g = kns.train.step(ctx, desc, p.detach(), batch)
    torch.cuda.synchronize()
    assert float(loss.detach()) == pytest.approx(float(parts[0]))
    # the weight gradients are sums of atomics: equal up to the order of FP32 additions
    g3 = 3.0 * g.cpu().numpy()
    np.testing.assert_allclose(p.grad.cpu().numpy(), g3, rtol=1e-4, atol=1e-5 * np.abs(g3).max())
    # a stale token is refused
    _, tok, _, _ = kns.train.forward(ctx, desc, p.detach(), batch)
    kns.train.forward(ctx, desc, p.detach(), batch)
    with pytest.raises(kns.KnsError):
        kns.train.backward(ctx, tok, p.detach())


def test_edge_cases(kns, ctx):
    desc = desc_of(2, 2)
    w = train_weights(desc, seed=2)
    params = torch.from_numpy(w).cuda()
    pr = problem(desc, 16, 8, 4, 8, seed=61)
    # rays that miss the box render black and cost |target|
    pr["o"][:4] = np.array([3.0, 3.0, 3.0], np.float32)
    pr["d"][:4] = np.array([1.0, 0.0, 0.0], np.float32)
    loss, tok, rgb, t = kns.train.forward(ctx, desc, params, gpu_batch(kns, pr), want_rgb=True, want_t=True)
    torch.cuda.synchronize()
    assert np.all(rgb.cpu().numpy()[:4] == 0) and np.all(t.cpu().numpy()[:4] == 0)
    _, parts_ref, _ = oracle.train_loss(desc, w, *oracle_args(pr))
    np.testing.assert_allclose(loss.cpu().numpy()[1:], parts_ref, rtol=2e-5)
    # no rays (eikonal only), no eikonal points, no importance samples
    for B, M, Ni in ((0, 8, 4), (16, 0, 4), (16, 8, 0)):
        q = problem(desc, max(B, 1), 8, max(Ni, 1), max(M, 1), seed=62)
        q = dict(o=q["o"][:B], d=q["d"][:B], target=q["target"][:B], u_s=q["u_s"][:B], u_i=q["u_i"][:B, :Ni],
                 P=q["P"][:M])
        loss, g = kns.train.step(ctx, desc, params, gpu_batch(kns, q))
        l_ref, parts_ref, g_ref = oracle.train_grad(desc, w, *oracle_args(q))
        np.testing.assert_allclose(loss.cpu().numpy()[1:], parts_ref, rtol=2e-5, atol=1e-9)
        if np.abs(g_ref).max() > 0:
            assert_grad_close(g.cpu().numpy().astype(np.float64), g_ref, rtol=2e-2, frac=0.99, norm_tol=1e-2)
    # bad arguments are refused on the host
    bad = gpu_batch(kns, pr)
    bad.u_strat = bad.u_strat[:, :1].contiguous()
    with pytest.raises(kns.KnsError):
        kns.train.forward(ctx, desc, params, bad)
    with pytest.raises(kns.KnsError):
        kns.train.forward(ctx, S.GridDesc(N=2, sdf_hidden=2, sdf_width=64, col_width=64, occ_res=0),
                          torch.zeros(8 * 20000, device="cuda"), gpu_batch(kns, pr))


def test_workload_architecture_small_batch(kns, ctx):
    """16^3 grid, 3 hidden layers, 64 + 32 samples, against the oracle with shared positions."""
    wl = S.TRAIN_WORKLOAD
    desc = desc_of(16, 3)
    w = train_weights(desc, seed=0)
    pr = problem(desc, 192, wl["n_strat"], wl["n_imp"], 256, seed=71, n_cams=8, W=32, H=32)
    args = oracle_args(pr, s=wl["s"], s_up=wl["s_up"], lam=wl["lam"], h=wl["h"])
    _, _, t_ref = oracle.train_loss(desc, w, *args, want_t=True)
    l_ref, parts_ref, g_ref = oracle.train_grad(desc, w, *args, t_fixed=t_ref)
    params = torch.from_numpy(w).cuda()
    loss, g = kns.train.step(ctx, desc, params, gpu_batch(kns, pr, s=wl["s"], s_up=wl["s_up"], lam=wl["lam"],
                                                            h=wl["h"], t_fixed=t_ref))
    np.testing.assert_allclose(loss.cpu().numpy()[1:], parts_ref, rtol=2e-5)
    assert_grad_close(g.cpu().numpy().astype(np.float64), g_ref, rtol=2e-3)


def test_full_size_workload_sampled(kns, ctx):
    """2^18 rays x (64 + 32) samples, 2^16 eikonal points on the 16^3 grid: sampled rays and the eikonal
    term against the oracle; the gradient against directional differences of the loss."""
    wl = S.TRAIN_WORKLOAD
    desc = desc_of(16, 3)
    w = train_weights(desc, seed=0)
    B, M = wl["n_rays"], wl["n_eik"]
    n_pix = wl["n_cams"] * wl["W"] * wl["H"]
    cams = S.orbit_cameras(wl["n_cams"], wl["W"], wl["H"], seed=1)
    sel, u_s, u_i, P = S.train_draws(B, wl["n_strat"], wl["n_imp"], M, n_pix, seed=0)
    o, d = S.pixel_rays(cams, wl["W"], wl["H"], sel)
    tdesc = desc_of(16, 3)
    tw = S.sal_sphere_grid(tdesc, seed=wl["target_seed"], perturb_std=wl["target_std"])
    tgt = oracle.render(tdesc, tw, None, cams, wl["W"], wl["H"], wl["max_steps"], wl["eps"], sel=sel)["rgb"]
    pr = dict(o=o, d=d, target=tgt, u_s=u_s, u_i=u_i, P=P)
    batch = gpu_batch(kns, pr, s=wl["s"], s_up=wl["s_up"], lam=wl["lam"], h=wl["h"])
    params = torch.from_numpy(w).cuda()
    loss, tok, rgb, t = kns.train.forward(ctx, desc, params, batch, want_rgb=True, want_t=True)
    g = kns.train.backward(ctx, tok, params)
    torch.cuda.synchronize()
    loss = loss.cpu().numpy().astype(np.float64)
    rgb = rgb.cpu().numpy()
    g = g.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(rgb))
    # the colour term is the mean L1 error of the returned colours
    assert loss[1] == pytest.approx(np.abs(rgb.astype(np.float64) - tgt).sum(1).mean(), rel=1e-5)
    # sampled rays rendered by the oracle with the same draws
    rs = np.random.default_rng(0).choice(B, 256, replace=False)
    sub = dict(o=o[rs], d=d[rs], target=tgt[rs], u_s=u_s[rs], u_i=u_i[rs], P=P[:0])
    _, _, t_ref, rgb_ref = oracle.train_loss(desc, w, *oracle_args(sub, s=wl["s"], s_up=wl["s_up"], lam=wl["lam"],
                                                                    h=wl["h"]), want_t=True, want_rgb=True)
    assert np.mean(np.abs(rgb[rs] - rgb_ref).max(1) <= 1e-4) >= 0.99
    assert np.mean(np.abs(t.cpu().numpy()[rs] - t_ref) <= 1e-4 * np.maximum(1.0, t_ref)) >= 0.99
    # the eikonal term over all 2^16 points
    eik = dict(o=o[:0], d=d[:0], target=tgt[:0], u_s=u_s[:0], u_i=u_i[:0], P=P)
    _, parts_eik, _ = oracle.train_loss(desc, w, *oracle_args(eik, s=wl["s"], s_up=wl["s_up"], lam=wl["lam"],
                                                              h=wl["h"]))
    assert loss[2] == pytest.approx(parts_eik[1], rel=2e-5)
    # directional differences of the GPU loss at fixed positions, along the colour weights and along
    # the SDF weights of the cells the samples touch
    fixed = gpu_batch(kns, pr, s=wl["s"], s_up=wl["s_up"], lam=wl["lam"], h=wl["h"], t_fixed=t.cpu().numpy())
    p_sdf = S.layer_offsets(desc)[len(desc.sdf_layers())][0]
    rng = np.random.default_rng(3)
    for part in ("colour", "sdf"):
        v = rng.normal(size=w.size).astype(np.float32).reshape(desc.n_cells, desc.p_cell)
        if part == "colour":
            v[:, :p_sdf] = 0
        else:
            v[:, p_sdf:] = 0
        v = v.reshape(-1)
        eps = 1e-3 / np.abs(v).max()
        lp = kns.train.forward(ctx, desc, params + eps * torch.from_numpy(v).cuda(), fixed)[0][0].item()
        lm = kns.train.forward(ctx, desc, params - eps * torch.from_numpy(v).cuda(), fixed)[0][0].item()
        fd = (lp - lm) / (2 * eps)
        assert float(g @ v.astype(np.float64)) == pytest.approx(fd, rel=2e-2), part
