"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test pins one part of the path to a closed form, a hand-derived value, an
exact identity of the method, or brute force:
  - the encoding of Eq. 1 against hand-evaluated sines and cosines;
  - softplus (Sec. 3.1) against its special values and symmetry;
  - the cell map m (Sec. 3.1) against hand-computed indices and tie rules;
  - the SDF MLP of Eq. 2 against an exact plane (softplus pair identity);
  - sphere tracing (Sec. 3.4.1) against the plane's closed-form step sequence;
  - the analytic normal against central finite differences on dense random grids;
  - the colour MLP of Eq. 3 against sigmoid(linear) routing of z, n and gamma(v);
  - the occupancy mask against the plane's closed form at voxel centres;
  - empty-space skipping against the closed-form plane root;
  - near-sphere renders against brute-force root marching.
"""
import math

import numpy as np
import pytest

import gridkit as K
import oracle as O
from paper_2206_10885_gb300 import synth as S

PI = math.pi


def small_desc(**kw):
    base = dict(N=4, sdf_hidden=3, sdf_width=32, col_width=32, occ_res=0)
    base.update(kw)
    return S.GridDesc(**base)


# ------------------------------------------------------------------ Eq. 1
def test_pe_hand_values():
    """gamma_4 at (0, 1/2, -1/4): raw xyz, then per k sin(2^k pi p) for xyz, cos for xyz."""
    r2 = math.sqrt(0.5)
    expect = [0.0, 0.5, -0.25,
              # k=0: sin(pi p), cos(pi p)
              0.0, 1.0, -r2, 1.0, 0.0, r2,
              # k=1: sin(2 pi p), cos(2 pi p)
              0.0, 0.0, -1.0, 1.0, -1.0, 0.0,
              # k=2: sin(4 pi p), cos(4 pi p)
              0.0, 0.0, 0.0, 1.0, 1.0, -1.0,
              # k=3: sin(8 pi p), cos(8 pi p)
              0.0, 0.0, 0.0, 1.0, 1.0, 1.0]
    got = O.pe(4, [0.0, 0.5, -0.25])
    assert got.shape == (27,)
    np.testing.assert_allclose(got, expect, atol=1e-15)


def test_pe_dimension_rule():
    """An R^n point maps to R^(n + 2nL) (Sec. 3.1)."""
    for L in range(0, 7):
        assert O.pe(L, [0.1, 0.2, 0.3]).size == 3 + 6 * L
    assert O.pe(2, [0.3]).size == 5


# --------------------------------------------------------------- softplus
def test_softplus_special_values():
    beta = 100.0
    assert O.softplus(0.0, beta) == pytest.approx(math.log(2.0) / beta, rel=1e-15)
    # far from zero it is the identity / zero to within exp(-beta|s|)/beta
    assert O.softplus(0.5, beta) == pytest.approx(0.5, abs=1e-22)
    assert O.softplus(-0.5, beta) == pytest.approx(0.0, abs=1e-23)
    # log(1 + e^(beta s))/beta at beta s = 1: log(1 + e)/100
    assert O.softplus(0.01, beta) == pytest.approx(math.log(1.0 + math.e) / 100.0, rel=1e-14)
    for s in np.linspace(-0.2, 0.2, 41):
        assert O.softplus(s, beta) - O.softplus(-s, beta) == pytest.approx(s, abs=1e-16)


# ------------------------------------------------------------------ m(x)
def test_cell_map_hand_values():
    d = small_desc(N=8)
    cases = {(-0.99, -0.99, -0.99): 0,
             (0.99, 0.99, 0.99): 511,
             (0.01, -0.01, 0.3): 4 + 8 * (3 + 8 * 5),
             (-1.0, -1.0, -1.0): 0,            # box face: clamped into the first cell
             (1.0, 1.0, 1.0): 511,             # far face: clamped into the last cell
             (0.0, 0.0, 0.0): 4 + 8 * (4 + 8 * 4),  # interior face: the higher cell
             (-0.75, 0.25, 0.5): 1 + 8 * (5 + 8 * 6),
             (1.5, -3.0, 0.1): 7 + 8 * (0 + 8 * 4)}  # outside: clamped per axis
    for x, c in cases.items():
        assert O.cell(d, x) == c, x


# ---------------------------------------------------------- Eq. 2 (plane)
A_PLANE = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
B_PLANE = 0.1


def f32(v):
    return np.asarray(v, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("hidden,width", [(2, 32), (3, 32), (3, 64)])
def test_sdf_exact_plane(hidden, width):
    d = small_desc(N=4, sdf_hidden=hidden, sdf_width=width, col_width=width)
    rng = np.random.default_rng(0)
    fc = rng.uniform(-2, 2, d.feat_dim)
    fe = rng.uniform(-1, 1, d.feat_dim)
    cb = rng.uniform(-0.3, 0.3, d.n_cells)
    w = K.plane_grid(d, A_PLANE, B_PLANE, feat_c=fc, feat_e=fe, cell_b=cb)
    a, fc32, fe32, cb32 = f32(A_PLANE), f32(fc), f32(fe), f32(cb)
    pts = rng.uniform(-1, 1, (400, 3))
    dd, feat, grad, cells = O.sdf(d, w, pts)
    s = pts @ a + cb32[cells]
    np.testing.assert_allclose(dd, s, atol=2e-15)
    np.testing.assert_allclose(feat, s[:, None] * fc32[None, :] + fe32[None, :], atol=1e-14)
    np.testing.assert_allclose(grad, np.broadcast_to(a, grad.shape), atol=1e-14)


def test_sdf_pe_column_pick():
    """A first layer that picks encoding column j makes d = gamma(x)[j] exactly."""
    d = small_desc(N=2, pe_pos_L=4)
    rng = np.random.default_rng(1)
    pts = rng.uniform(-1, 1, (50, 3))
    for col in range(d.sdf_in):
        w = K.pe_pick_grid(d, col)
        dd, _, grad, _ = O.sdf(d, w, pts)
        if col < 3:
            want, gw = pts[:, col], np.eye(3)[col][None, :].repeat(len(pts), 0)
        else:
            k, r = divmod(col - 3, 6)
            c = r % 3
            f = (2 ** k) * PI
            if r < 3:
                want = np.sin(f * pts[:, c])
                gcomp = f * np.cos(f * pts[:, c])
            else:
                want = np.cos(f * pts[:, c])
                gcomp = -f * np.sin(f * pts[:, c])
            gw = np.zeros((len(pts), 3))
            gw[:, c] = gcomp
        np.testing.assert_allclose(dd, want, atol=1e-13, err_msg=str(col))
        np.testing.assert_allclose(grad, gw, atol=1e-11, err_msg=str(col))


# ------------------------------------------------- Sec. 3.4.1 (plane trace)
def slab(o, w):
    tn, tf = -np.inf, np.inf
    for k in range(3):
        t1, t2 = (-1 - o[k]) / w[k], (1 - o[k]) / w[k]
        tn, tf = max(tn, min(t1, t2)), min(tf, max(t1, t2))
    return max(tn, 0.0), tf


def plane_rays(n, seed, a, b):
    rng = np.random.default_rng(seed)
    os_, ws = [], []
    while len(os_) < n:
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        o = 2.5 * u
        if o @ a + b <= 0.2:
            continue
        tgt = rng.uniform(-0.4, 0.4, 3)
        tgt -= (tgt @ a + b) * a  # project onto the plane
        w = tgt - o
        w /= np.linalg.norm(w)
        os_.append(o)
        ws.append(w)
    return np.array(os_), np.array(ws)


def closed_form_trace(o, w, a, b, eps, max_steps):
    t0, tf = slab(o, w)
    r = 1.0 + a @ w
    d0 = a @ (o + t0 * w) + b
    t, dk = t0, d0
    for k in range(max_steps):
        if abs(dk) < eps:
            return t0 + d0 * (1 - r ** k) / (1 - r), k + 1, abs(abs(dk) - eps)
        t, dk = t + dk, dk * r
        if t > tf:
            return np.inf, k + 1, None
    return np.inf, max_steps, None


@pytest.mark.parametrize("eps", [1e-4, 1e-3])
def test_sphere_trace_plane_closed_form(eps):
    d = small_desc(N=4)
    w = K.plane_grid(d, A_PLANE, B_PLANE)
    a, b = f32(A_PLANE), float(np.float32(B_PLANE))
    o, ws = plane_rays(300, 3, a, b)
    out = O.trace_rays(d, w, None, o, ws, 200, eps)
    checked = 0
    for q in range(len(o)):
        t_cf, steps_cf, margin = closed_form_trace(o[q], ws[q], a, b, eps, 200)
        if margin is None or margin < 1e-9:
            continue
        checked += 1
        assert out["steps"][q] == steps_cf
        assert out["depth"][q] == pytest.approx(t_cf, abs=1e-12)
        np.testing.assert_allclose(out["normal"][q], a / np.linalg.norm(a), atol=1e-14)
        # the hit is within eps / cos(incidence) of the true root
        t_root = -(a @ o[q] + b) / (a @ ws[q])
        assert abs(out["depth"][q] - t_root) <= eps / abs(a @ ws[q]) + 1e-12
    assert checked > 250


def test_trace_normal_incidence_one_step():
    """Along -a the plane SDF is the exact distance: the second evaluation lands on it."""
    d = small_desc(N=4)
    w = K.plane_grid(d, A_PLANE, B_PLANE)
    a, b = f32(A_PLANE), float(np.float32(B_PLANE))
    an = a / np.linalg.norm(a)
    o = 3.0 * an - b * an + np.array([0.01, -0.02, 0.0]) @ (np.eye(3) - np.outer(an, an))
    out = O.trace_rays(d, w, None, o[None], -an[None], 10, 1e-6)
    assert out["steps"][0] == 2
    t0, _ = slab(o, -an)
    d0 = a @ (o - t0 * an) + b
    assert out["depth"][0] == pytest.approx(t0 + d0, abs=1e-12)
    assert out["depth"][0] == pytest.approx(-(a @ o + b) / (a @ -an), abs=1e-6)


def test_trace_misses_and_edges():
    d = small_desc(N=4)
    w = K.plane_grid(d, A_PLANE, B_PLANE)
    # ray that misses the box entirely
    o = np.array([[3.0, 3.0, 3.0]])
    out = O.trace_rays(d, w, None, o, np.array([[1.0, 0.0, 0.0]]), 64, 1e-4)
    assert out["depth"][0] == np.inf and out["cell"][0] == -1 and out["steps"][0] == 0
    # a ray parallel to the plane never hits: it leaves through the far face
    perp = np.cross(A_PLANE, [0, 0, 1.0])
    perp /= np.linalg.norm(perp)
    o = -2.0 * perp + 0.5 * A_PLANE
    out = O.trace_rays(d, w, None, o[None], perp[None], 64, 1e-4)
    assert out["depth"][0] == np.inf and out["cell"][0] == -1
    # a budget of one step: hit only if the entry point is already on the surface
    a, b = f32(A_PLANE), float(np.float32(B_PLANE))
    o, ws = plane_rays(20, 5, a, b)
    out = O.trace_rays(d, w, None, o, ws, 1, 1e-4)
    assert np.all(out["steps"] == 1) and np.all(np.isinf(out["depth"]))
    # camera inside the box: tracing starts at t = 0
    o = np.array([[0.5, 0.5, 0.5]])
    dirv = -A_PLANE[None]
    out = O.trace_rays(d, w, None, o, dirv, 64, 1e-6)
    t_root = (a @ o[0] + b)
    assert out["depth"][0] == pytest.approx(t_root, abs=1e-6)
    # axis-parallel ray (two zero direction components)
    o = np.array([[2.0, 0.1, 0.2]])
    out = O.trace_rays(d, w, None, o, np.array([[-1.0, 0.0, 0.0]]), 200, 1e-6)
    root = 2.0 + (a[1] * 0.1 + a[2] * 0.2 + b) / a[0]
    assert out["depth"][0] == pytest.approx(root, abs=1e-5)
    # a ray that enters on the negative side steps backwards out of the interval: a miss
    out = O.trace_rays(d, w, None, -o, np.array([[1.0, 0.0, 0.0]]), 200, 1e-6)
    assert out["depth"][0] == np.inf and out["steps"][0] == 1


# ----------------------------------------------------- normals (FD pin)
@pytest.mark.parametrize("L,width,hidden", [(4, 32, 2), (4, 32, 3), (6, 64, 3)])
def test_gradient_matches_central_differences(L, width, hidden):
    d = small_desc(N=4, pe_pos_L=L, sdf_width=width, col_width=width, sdf_hidden=hidden,
                   softplus_beta=10.0)
    w = K.random_grid(d, seed=L + width, scale=0.4)
    rng = np.random.default_rng(7)
    pts = rng.uniform(-0.95, 0.95, (200, 3))
    # keep points whose +-h neighbourhood stays inside one cell
    u = (pts + 1) * d.N / 2
    ok = np.all(np.abs(u - np.round(u)) > 1e-3, axis=1)
    pts = pts[ok]
    _, _, grad, cells = O.sdf(d, w, pts)
    h = 1e-6
    fd = np.zeros_like(grad)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        dp = np.array([O.sdf_cell(d, w, cl, p + e, False, False)[0] for p, cl in zip(pts, cells)])
        dm = np.array([O.sdf_cell(d, w, cl, p - e, False, False)[0] for p, cl in zip(pts, cells)])
        fd[:, c] = (dp - dm) / (2 * h)
    scale = np.maximum(1.0, np.abs(grad))
    assert np.max(np.abs(fd - grad) / scale) < 2e-6


def test_gradient_plane_through_random_features():
    """The gradient ignores the feature rows: a plane d with random z rows keeps grad = a."""
    d = small_desc(N=2)
    rng = np.random.default_rng(3)
    w = K.plane_grid(d, A_PLANE, B_PLANE, feat_c=rng.normal(size=d.feat_dim) * 5)
    _, _, grad, _ = O.sdf(d, w, rng.uniform(-1, 1, (20, 3)))
    np.testing.assert_allclose(grad, np.broadcast_to(f32(A_PLANE), grad.shape), atol=1e-13)


# --------------------------------------------------------- Eq. 3 (colour)
def test_colour_linear_routing():
    """RGB = sigmoid(K u_sel + b): z_0, z_14, n, raw v, sin(pi v_x), cos(2 pi v_z)."""
    d = small_desc(N=4, pe_dir_L=2)
    rng = np.random.default_rng(11)
    fc = rng.uniform(-1, 1, d.feat_dim)
    fe = rng.uniform(-1, 1, d.feat_dim)
    w = K.plane_grid(d, A_PLANE, B_PLANE, feat_c=fc, feat_e=fe)
    F = d.feat_dim
    # colour input u = [z (15), n (3), gamma_2(v) (15)]
    g0 = F + 3
    sel = [0, 14, F + 0, F + 1, F + 2, g0 + 0, g0 + 1, g0 + 2, g0 + 3, g0 + 3 + 6 + 5]
    Km = rng.uniform(-1, 1, (3, len(sel)))
    bias = rng.uniform(-0.5, 0.5, 3)
    w = K.set_colour_linear(d, w, sel, Km, bias)
    a, b = f32(A_PLANE), float(np.float32(B_PLANE))
    o, ws = plane_rays(40, 9, a, b)
    out = O.trace_rays(d, w, None, o, ws, 200, 1e-5)
    assert np.all(np.isfinite(out["depth"]))
    Kf, bf = f32(Km), f32(bias)
    for q in range(len(o)):
        x = o[q] + out["depth"][q] * ws[q]
        s = a @ x + b
        z = s * f32(fc) + f32(fe)
        n = a / np.linalg.norm(a)
        v = ws[q]
        vals = [z[0], z[14], n[0], n[1], n[2], v[0], v[1], v[2], math.sin(PI * v[0]), math.cos(2 * PI * v[2])]
        want = K.sigmoid(Kf @ np.array(vals) + bf)
        np.testing.assert_allclose(out["rgb"][q], want, atol=1e-13)


def test_colour_includes_x_when_flagged():
    d = small_desc(N=4, col_use_x=1)
    w = K.plane_grid(d, A_PLANE, B_PLANE)
    base = d.feat_dim + 3 + 3 + 6 * d.pe_dir_L
    Km = np.array([[1.0, 0, 0], [0, -2.0, 0], [0, 0, 0.5]])
    w = K.set_colour_linear(d, w, [base, base + 1, base + 2], Km, [0, 0, 0])
    x = np.array([0.3, -0.2, 0.6])
    rgb = O.colour(d, w, 5, x, np.zeros(d.feat_dim), [0, 0, 1], [1, 0, 0])
    np.testing.assert_allclose(rgb, K.sigmoid([0.3, 0.4, 0.3]), atol=1e-15)


def test_colour_cell_map_through_image():
    """Per-cell colour bias: RGB = sigmoid(bias[cell]) identifies the hit cell (Sec. 3.1)."""
    d = small_desc(N=8)
    cb = np.zeros((d.n_cells, 3))
    ids = np.arange(d.n_cells)
    cb[:, 0] = (ids % 8) * 0.25 - 1.0
    cb[:, 1] = ((ids // 8) % 8) * 0.25 - 1.0
    cb[:, 2] = (ids // 64) * 0.25 - 1.0
    w = K.plane_grid(d, A_PLANE, B_PLANE)
    w = K.set_colour_linear(d, w, [0], np.zeros((3, 1)), [0, 0, 0], cell_bias=cb)
    a, b = f32(A_PLANE), float(np.float32(B_PLANE))
    o, ws = plane_rays(200, 13, a, b)
    out = O.trace_rays(d, w, None, o, ws, 200, 1e-6)
    for q in range(len(o)):
        x = o[q] + out["depth"][q] * ws[q]
        idx = np.floor((x + 1) * 4)
        if np.any(np.abs((x + 1) * 4 - np.round((x + 1) * 4)) < 1e-6):
            continue
        c = int(idx[0] + 8 * (idx[1] + 8 * idx[2]))
        assert out["cell"][q] == c
        logit = np.log(out["rgb"][q] / (1 - out["rgb"][q]))
        got = np.round((logit + 1.0) / 0.25).astype(int)
        assert got[0] + 8 * (got[1] + 8 * got[2]) == c


# ------------------------------------------------------------- occupancy
def test_occupancy_plane_closed_form():
    d = small_desc(N=4, occ_res=32)
    w = K.plane_grid(d, A_PLANE, B_PLANE)
    bits = O.occupancy(d, w, 32)
    a, b = f32(A_PLANE), float(np.float32(B_PLANE))
    c = -1 + (np.arange(32) + 0.5) * (2 / 32)
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    val = np.abs(a[0] * X + a[1] * Y + a[2] * Z + b)
    diag = math.sqrt(3) * 2 / 32
    want = (val < diag).transpose(2, 1, 0).reshape(-1)  # x fastest
    got = np.unpackbits(bits.view(np.uint8), bitorder="little")[:32 ** 3].astype(bool)
    ok = np.abs(val - diag).transpose(2, 1, 0).reshape(-1) > 1e-12
    assert np.array_equal(got[ok], want[ok])
    assert want.sum() > 100


@pytest.mark.parametrize("res", [16, 32])
def test_empty_space_skip_plane(res):
    """With the mask, the trace jumps to the band and still lands within eps/cos of the root."""
    d = small_desc(N=4, occ_res=res)
    w = K.plane_grid(d, A_PLANE, B_PLANE)
    occ = O.occupancy(d, w, res)
    a, b = f32(A_PLANE), float(np.float32(B_PLANE))
    o, ws = plane_rays(300, 21, a, b)
    eps = 1e-5
    with_occ = O.trace_rays(d, w, occ, o, ws, 200, eps)
    without = O.trace_rays(d, w, None, o, ws, 200, eps)
    t_root = np.array([-(a @ o[q] + b) / (a @ ws[q]) for q in range(len(o))])
    bound = eps / np.abs(ws @ a) + 1e-12
    assert np.all(np.abs(with_occ["depth"] - t_root) <= bound)
    assert np.all(with_occ["steps"] <= without["steps"])
    assert np.mean(with_occ["steps"]) < np.mean(without["steps"])


def test_empty_mask_misses_everything():
    d = small_desc(N=4, occ_res=16)
    w = K.plane_grid(d, A_PLANE, B_PLANE)
    occ = np.zeros((16 ** 3 + 63) // 64, dtype=np.uint64)
    a, b = f32(A_PLANE), float(np.float32(B_PLANE))
    o, ws = plane_rays(50, 2, a, b)
    out = O.trace_rays(d, w, occ, o, ws, 64, 1e-4)
    assert np.all(np.isinf(out["depth"])) and np.all(out["steps"] == 0)


def test_full_mask_equals_no_mask():
    d = small_desc(N=4, occ_res=16)
    w = K.plane_grid(d, A_PLANE, B_PLANE)
    occ = np.full((16 ** 3 + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    a, b = f32(A_PLANE), float(np.float32(B_PLANE))
    o, ws = plane_rays(100, 4, a, b)
    r1 = O.trace_rays(d, w, occ, o, ws, 64, 1e-4)
    r2 = O.trace_rays(d, w, None, o, ws, 64, 1e-4)
    assert np.array_equal(r1["depth"], r2["depth"]) and np.array_equal(r1["steps"], r2["steps"])


def test_dda_matches_fine_sampling():
    """The DDA's next occupied voxel and entry t agree with sampling the ray every 1e-5."""
    res = 16
    d = small_desc(N=4, occ_res=res)
    rng = np.random.default_rng(5)
    occ_bool = rng.uniform(size=res ** 3) < 0.02
    words = np.packbits(occ_bool.astype(np.uint8), bitorder="little").view(np.uint64)
    checked = 0
    for q in range(60):
        o = rng.normal(size=3)
        o = 2.5 * o / np.linalg.norm(o)
        tgt = rng.uniform(-0.6, 0.6, 3)
        wv = (tgt - o) / np.linalg.norm(tgt - o)
        t0, tf = slab(o, wv)
        ts = np.arange(t0, tf, 1e-5)
        xs = o[None, :] + ts[:, None] * wv[None, :]
        idx = np.clip(np.floor((xs + 1) * res / 2).astype(int), 0, res - 1)
        lin = idx[:, 0] + res * (idx[:, 1] + res * idx[:, 2])
        hitmask = occ_bool[lin]
        start_empty = not hitmask[0]
        if not start_empty:
            continue
        got = O.first_occupied(d, words, o, wv, t0)
        if not hitmask.any():
            assert got is None
            continue
        k = int(np.argmax(hitmask))
        assert got is not None
        assert tuple(idx[k]) == got[1]
        assert ts[k - 1] - 1e-12 <= got[0] <= ts[k] + 1e-12
        checked += 1
    assert checked > 20


# ---------------------------------------------- brute force (near-sphere)
def test_near_sphere_hits_match_brute_force_roots():
    desc, w, cams, W, H, ms, eps = S.workload("c1")
    # a tiny 16x16 image from each camera
    cams = S.orbit_cameras(4, 16, 16, seed=1, evenly_spaced=True)
    n = 4 * 16 * 16
    r = O.render(desc, w, None, cams, 16, 16, 256, eps)
    rays = [O.ray(cams[q // 256], (q % 256) // 16, q % 16) for q in range(n)]
    o = np.array([x[0] for x in rays])
    dirs = np.array([x[1] for x in rays])
    t0 = np.array([slab(o[q], dirs[q])[0] for q in range(n)])
    t1 = np.array([slab(o[q], dirs[q])[1] for q in range(n)])
    roots = O.march_roots(desc, w, o, dirs, t0, t1, 1e-4, 1e-12)
    hit = r["hit"] == 1
    assert hit.sum() > 40
    # every converged ray lands within |d|/|grad d . w| <= eps/|grad d . w| of a brute-force root
    # (first order), or past the first root when a step jumped a thin part (reported, not an error)
    both = hit & np.isfinite(roots)
    xh = o + r["depth"][:, None].astype(np.float64) * dirs
    _, _, g, _ = O.sdf(desc, w, xh)
    gdotw = np.abs(np.sum(g * dirs, axis=1))
    close = np.abs(r["depth"] - roots) <= 1.5 * eps / np.maximum(gdotw, 1e-3) + 2e-6
    later = r["depth"] > roots + 1e-6
    assert np.mean(close[both]) > 0.97
    assert np.sum(~close[both] & ~later[both]) == 0
    # rays the brute force says have no root must not report a hit
    assert not np.any(hit & ~np.isfinite(roots))


def test_conditioning_margins_only_shrink():
    """Conditioning-aware margins (a test-harness aid) never exceed the raw ones, and vanish at
    delta 0: the decisions and outputs themselves do not change."""
    desc, w, cams, W, H, ms, eps = S.workload("c1")
    cams = cams[:1]
    r0 = O.render(desc, w, None, cams, 24, 24, ms, eps)
    r1 = O.render(desc, w, None, cams, 24, 24, ms, eps, delta_step=2e-6)
    for k in ("rgb", "depth", "normal", "cell", "hit", "steps"):
        assert np.array_equal(r0[k], r1[k]), k
    m0, m1 = r0["margins"], r1["margins"]
    fin = np.isfinite(m0)
    assert np.all(m1[fin] <= m0[fin] + 1e-15)
