"""Near-sphere pin: the geometric (SAL) initialisation through the oracle's SDF MLP.

The workloads initialise every cell's SDF MLP (Eq. 2) geometrically, as SAL does, for a
sphere of radius r = 0.5: hidden weights N(0, 2/out), zero biases, only the raw xyz columns
of the encoding live in the first layer, the d row of the last layer at mean sqrt(pi)/sqrt(in)
with bias -r.  With ReLU units and infinite width that network computes |x| - r exactly; with
the softplus of Sec. 3.1 (beta = 100) and finite width it is a near-sphere whose radius is
fixed by the construction.  These tests pin the construction (synth.sal_sphere_grid) and the
oracle's SDF evaluation (ko_sdf_eval) together against a computation that shares nothing with
either: the infinite-width limit of the initialisation, a one-dimensional Gaussian recursion
evaluated by quadrature here.

Layer l's pre-activations are N(0, 2 q_{l-1}) with q_0 = |x|^2 / n (width n), and
q_l = E[softplus(z)^2]; the output is sqrt(pi n) E[softplus(z_L)] - r.  Its root r* is the
"known radius": exactly 0.5 in the ReLU limit, and smaller at beta = 100 because softplus
adds a positive offset of up to ln 2 / beta near zero.  A random draw of width 256 differs from
the limit by finite-width fluctuations of a few hundredths (measured over seeds 0..5: mean
radial root 0.45..0.50 at beta = 100, 0.50..0.56 in the ReLU limit), so the tolerance is 0.06.
A wrong sign of the d bias leaves no root; a dropped sqrt(2) scales the radius by 2^(H/2); a
wrong mean of the d row scales it by that factor; a wrong softplus offset moves r* by ~0.05 --
each fails here.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2206_10885_gb300 import synth as S

WIDTH = 256  # the widest MLP the oracle evaluates
TOL = 0.06


def fibonacci_dirs(n: int) -> np.ndarray:
    """n near-uniform unit directions (Fibonacci lattice on the sphere)."""
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = math.pi * (1.0 + math.sqrt(5.0)) * i
    r = np.sqrt(1.0 - z * z)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def radial_roots(desc, w, u: np.ndarray, r0: float = 0.5):
    """Root r(u) of d(r u) along each direction by Newton steps on the oracle's d and grad d,
    then checked as a sign change of d across r +- 1e-9.  Returns (r, |grad d| at r)."""
    r = np.full(len(u), r0)
    for _ in range(40):
        d, _, g, _ = O.sdf(desc, w, r[:, None] * u)
        step = d / np.sum(g * u, axis=1)
        r = r - step
        if np.max(np.abs(step)) < 1e-13:
            break
    lo, _, _, _ = O.sdf(desc, w, (r - 1e-9)[:, None] * u)
    hi, g, gr, _ = O.sdf(desc, w, (r + 1e-9)[:, None] * u)
    assert np.all(lo < 0) and np.all(hi > 0), "not a sign change from inside to outside"
    return r, np.linalg.norm(gr, axis=1)


def softplus(z, beta):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-beta * np.abs(z))) / beta


def gauss_expect(f, var: float) -> float:
    s = math.sqrt(var)
    z = np.linspace(-12.0 * s, 12.0 * s, 40001)
    pdf = np.exp(-0.5 * (z / s) ** 2) / (s * math.sqrt(2.0 * math.pi))
    return float(np.trapezoid(f(z) * pdf, z))


def limit_sdf(rho: float, n: int, hidden: int, beta: float, radius: float = 0.5) -> float:
    """d at distance rho from the centre for the infinite-width SAL network."""
    var = 2.0 * rho * rho / n
    m = 0.0
    for _ in range(hidden):
        m = gauss_expect(lambda z: softplus(z, beta), var)
        var = 2.0 * gauss_expect(lambda z: softplus(z, beta) ** 2, var)
    return math.sqrt(math.pi * n) * m - radius


def limit_radius(n: int, hidden: int, beta: float) -> float:
    lo, hi = 0.05, 1.5
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        if limit_sdf(mid, n, hidden, beta) < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def sal_single_cell(hidden: int, beta: float, seed: int):
    desc = S.GridDesc(N=1, sdf_hidden=hidden, sdf_width=WIDTH, col_width=32, occ_res=0, softplus_beta=beta)
    return desc, S.sal_sphere_grid(desc, seed=seed, perturb_std=0.0)


def test_limit_recursion_is_the_sphere_for_relu():
    """The recursion itself: in the ReLU limit it reproduces |x| - r at every depth and width."""
    for n in (32, 256):
        for h in (1, 2, 3):
            for rho in (0.25, 0.5, 0.9):
                assert abs(limit_sdf(rho, n, h, 1e7) - (rho - 0.5)) < 2e-5
    assert abs(limit_radius(256, 3, 1e7) - 0.5) < 1e-5


def test_near_sphere_radius_workload_softplus():
    """beta = 100, 3 hidden layers of width 256: mean radial root over 10^4 Fibonacci directions
    near r* of the limit, a narrow spread, and |grad d| near 1 at the surface (an SDF)."""
    r_star = limit_radius(WIDTH, 3, 100.0)
    assert 0.40 < r_star < 0.48  # the softplus offset shrinks the ReLU radius 0.5
    u = fibonacci_dirs(10000)
    desc, w = sal_single_cell(3, 100.0, seed=0)
    r, gn = radial_roots(desc, w, u)
    print("SAL width 256, 3 hidden, beta 100: r* = %.4f, mean r = %.4f, sd %.4f, range %.4f..%.4f, "
          "|grad d| %.3f..%.3f (mean %.3f)" % (r_star, r.mean(), r.std(), r.min(), r.max(), gn.min(), gn.max(),
                                               gn.mean()))
    assert abs(r.mean() - r_star) < TOL
    assert r.std() < 0.1
    assert 0.5 < gn.min() and gn.max() < 1.6 and abs(gn.mean() - 1.0) < 0.2


@pytest.mark.parametrize("hidden", [2, 3])
def test_near_sphere_radius_over_seeds(hidden):
    """Seeds 0..3 at both depths: every seed's mean root within 2 TOL of r*, their average within TOL."""
    u = fibonacci_dirs(2000)
    for beta in (100.0, 1e7):  # the workloads' softplus, and the ReLU limit where r* = 0.5 exactly
        r_star = limit_radius(WIDTH, hidden, beta)
        means = []
        for seed in range(4):
            desc, w = sal_single_cell(hidden, beta, seed)
            r, _ = radial_roots(desc, w, u)
            means.append(r.mean())
        assert all(abs(m - r_star) < 2 * TOL for m in means), (beta, r_star, means)
        assert abs(np.mean(means) - r_star) < TOL, (beta, r_star, means)


def test_near_sphere_pin_fails_on_planted_mistakes():
    """The pin is sensitive: the same check on deliberately broken constructions fails."""
    desc, w = sal_single_cell(3, 100.0, seed=0)
    r_star = limit_radius(WIDTH, 3, 100.0)
    u = fibonacci_dirs(400)
    layers = S.layer_offsets(desc)
    # (a) the d bias with the wrong sign: d > 0 everywhere near the centre, no inside
    bad = w.copy()
    _, b_off, _, _ = layers[len(desc.sdf_layers()) - 1]
    bad[b_off] = +0.5
    d0, _, _, _ = O.sdf(desc, bad, np.zeros((1, 3)))
    assert d0[0] > 0
    # (b) hidden layers without the sqrt(2) of the He scale: the radius grows by ~2^(H/2)
    bad = w.copy()
    for li in range(1, desc.sdf_hidden):
        w_off, b_off, i, o = layers[li]
        bad[w_off:b_off] /= math.sqrt(2.0)
    r, _ = radial_roots(desc, bad, u, r0=1.0)
    assert abs(r.mean() - r_star) > 3 * TOL
    # (c) the d row's mean sqrt(pi)/sqrt(in) replaced by sqrt(pi)/in
    bad = w.copy()
    w_off, b_off, i, o = layers[len(desc.sdf_layers()) - 1]
    bad[w_off:w_off + i] /= math.sqrt(i)
    d_far, _, _, _ = O.sdf(desc, bad, np.array([[0.99, 0.0, 0.0]]))
    assert d_far[0] < 0  # still inside at the box face: the radius grew by sqrt(in) = 16
