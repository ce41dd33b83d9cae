"""Pins for the oracle's Gaussian overlap cost and its adjoint.

Each pin holds the oracle to something other than itself: a second
formulation (expanded squared distance, numpy, FP64), the closed form of two
single Gaussians checked by grid quadrature of the product of two normal
densities, exact symmetries and invariances of the cost, and central finite
differences for the analytic gradient.
"""
import numpy as np
import pytest

import synth


def _tiny_clouds(rng, n, dim, max_pts=5, grid=None):
    sizes = rng.integers(1, max_pts + 1, size=n)
    off = np.zeros(n + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    tot = int(off[-1])
    pts = rng.uniform(-0.3, 0.3, size=(tot, dim))
    if grid is not None:
        pts = np.round(pts / grid) * grid
    return {"dim": dim, "offsets": off,
            "x": pts[:, 0].astype(np.float32), "y": pts[:, 1].astype(np.float32),
            "z": pts[:, 2].astype(np.float32) if dim == 3 else None,
            "sigma": rng.uniform(0.05, 0.15, size=tot).astype(np.float32),
            "weight": rng.uniform(0.5, 2.0, size=tot).astype(np.float32)}


def _expanded_form(c, i, j, params=None):
    """f written with |u-v|^2 = |u|^2 + |v|^2 - 2 u.v and a matrix product."""
    sl_i = slice(c["offsets"][i], c["offsets"][i + 1])
    sl_j = slice(c["offsets"][j], c["offsets"][j + 1])
    cols = ["x", "y"] + (["z"] if c["dim"] == 3 else [])
    A = np.stack([c[k][sl_i].astype(np.float64) for k in cols], 1)
    B = np.stack([c[k][sl_j].astype(np.float64) for k in cols], 1)
    if params is not None:
        th, tx, ty = params
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        B = B @ R.T + np.array([tx, ty])
    d2 = (A * A).sum(1)[:, None] + (B * B).sum(1)[None, :] - 2.0 * A @ B.T
    sa = c["sigma"][sl_i].astype(np.float64)
    sb = c["sigma"][sl_j].astype(np.float64)
    s2 = sa[:, None] ** 2 + sb[None, :] ** 2
    wa = c["weight"][sl_i].astype(np.float64)
    wb = c["weight"][sl_j].astype(np.float64)
    return float((wa[:, None] * wb[None, :] * np.exp(-d2 / (2.0 * s2))).sum())


@pytest.mark.parametrize("dim", [2, 3])
def test_overlap_matches_expanded_form(oracle_lib, dim):
    rng = np.random.default_rng(11 + dim)
    c = _tiny_clouds(rng, 8, dim)
    pi, pj = oracle_lib.all_pairs(8)
    f = oracle_lib.overlap(c, pi, pj, n_threads=2)
    ref = np.array([_expanded_form(c, i, j) for i, j in zip(pi, pj)])
    np.testing.assert_allclose(f, ref, rtol=1e-12, atol=0)


def test_overlap_with_transform_matches_expanded_form(oracle_lib):
    rng = np.random.default_rng(5)
    c = _tiny_clouds(rng, 6, 2)
    pi, pj = oracle_lib.all_pairs(6)
    params = np.stack([rng.uniform(-np.pi, np.pi, len(pi)),
                       rng.uniform(-0.2, 0.2, len(pi)),
                       rng.uniform(-0.2, 0.2, len(pi))], 1)
    f = oracle_lib.overlap(c, pi, pj, params=params, n_threads=1)
    ref = np.array([_expanded_form(c, i, j, p) for i, j, p in zip(pi, pj, params)])
    np.testing.assert_allclose(f, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("dim", [2, 3])
def test_single_points_closed_form_and_quadrature(oracle_lib, dim):
    # f of two single points = w_a w_b exp(-D^2 / (2 (sa^2 + sb^2)))
    xa, xb = np.array([0.11, -0.05, 0.02]), np.array([-0.07, 0.08, -0.03])
    sa, sb, wa, wb = 0.09, 0.06, 1.5, 0.75
    c = {"dim": dim, "offsets": np.array([0, 1, 2], np.int64),
         "x": np.array([xa[0], xb[0]], np.float32), "y": np.array([xa[1], xb[1]], np.float32),
         "z": np.array([xa[2], xb[2]], np.float32) if dim == 3 else None,
         "sigma": np.array([sa, sb], np.float32), "weight": np.array([wa, wb], np.float32)}
    f = oracle_lib.overlap(c, [0], [1], n_threads=1)[0]
    pa = np.array([c["x"][0], c["y"][0]] + ([c["z"][0]] if dim == 3 else []), np.float64)
    pb = np.array([c["x"][1], c["y"][1]] + ([c["z"][1]] if dim == 3 else []), np.float64)
    sa2, sb2 = float(np.float32(sa)) ** 2, float(np.float32(sb)) ** 2
    w = float(np.float32(wa)) * float(np.float32(wb))
    closed = w * np.exp(-((pa - pb) ** 2).sum() / (2 * (sa2 + sb2)))
    assert abs(f - closed) <= 1e-14 * closed
    if dim == 2:
        # reading check: f = w (2 pi s2)^{d/2} * integral of N(x; xa, sa2 I) N(x; xb, sb2 I)
        h = 0.002
        g = np.arange(-0.8, 0.8, h)
        X, Y = np.meshgrid(g, g, indexing="ij")
        na = np.exp(-((X - pa[0]) ** 2 + (Y - pa[1]) ** 2) / (2 * sa2)) / (2 * np.pi * sa2)
        nb = np.exp(-((X - pb[0]) ** 2 + (Y - pb[1]) ** 2) / (2 * sb2)) / (2 * np.pi * sb2)
        integral = (na * nb).sum() * h * h
        quad = w * (2 * np.pi * (sa2 + sb2)) * integral
        assert abs(f - quad) <= 1e-8 * f


@pytest.mark.parametrize("dim", [2, 3])
def test_overlap_symmetric_at_identity(oracle_lib, dim):
    rng = np.random.default_rng(3)
    c = _tiny_clouds(rng, 7, dim)
    pi, pj = oracle_lib.all_pairs(7)
    f1 = oracle_lib.overlap(c, pi, pj, n_threads=2)
    f2 = oracle_lib.overlap(c, pj, pi, n_threads=2)
    np.testing.assert_allclose(f1, f2, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dim", [2, 3])
def test_overlap_translation_and_quarter_turn_invariant(oracle_lib, dim):
    rng = np.random.default_rng(4)
    grid = 2.0 ** -12            # coordinates on a grid so the moves are exact in FP32
    c = _tiny_clouds(rng, 6, dim, grid=grid)
    pi, pj = oracle_lib.all_pairs(6)
    f0 = oracle_lib.overlap(c, pi, pj, n_threads=2)
    shifted = dict(c)
    shifted["x"] = (c["x"] + np.float32(0.375)).astype(np.float32)
    shifted["y"] = (c["y"] - np.float32(0.25)).astype(np.float32)
    if dim == 3:
        shifted["z"] = (c["z"] + np.float32(0.125)).astype(np.float32)
    np.testing.assert_allclose(oracle_lib.overlap(shifted, pi, pj, n_threads=2), f0,
                               rtol=1e-12, atol=0)
    turned = dict(c)                      # (x, y) -> (-y, x) on both clouds
    turned["x"] = (-c["y"]).astype(np.float32)
    turned["y"] = c["x"].copy()
    np.testing.assert_allclose(oracle_lib.overlap(turned, pi, pj, n_threads=2), f0,
                               rtol=1e-12, atol=0)


def test_transform_equals_moved_cloud(oracle_lib):
    # f(i, j; theta = pi/2, t) = f at identity with item j moved by the same map
    rng = np.random.default_rng(8)
    grid = 2.0 ** -12
    c = _tiny_clouds(rng, 2, 2, grid=grid)
    t = (0.125, -0.0625)
    f = oracle_lib.overlap(c, [0], [1], params=np.array([[np.pi / 2, t[0], t[1]]]))[0]
    moved = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in c.items()}
    sl = slice(c["offsets"][1], c["offsets"][2])
    moved["x"][sl] = (-c["y"][sl] + np.float32(t[0])).astype(np.float32)
    moved["y"][sl] = (c["x"][sl] + np.float32(t[1])).astype(np.float32)
    g = oracle_lib.overlap(moved, [0], [1])[0]
    assert abs(f - g) <= 1e-12 * g


def test_gradient_matches_central_differences(oracle_lib):
    rng = np.random.default_rng(21)
    c = _tiny_clouds(rng, 5, 2)
    pi, pj = oracle_lib.all_pairs(5)
    params = np.stack([rng.uniform(-0.5, 0.5, len(pi)), rng.uniform(-0.1, 0.1, len(pi)),
                       rng.uniform(-0.1, 0.1, len(pi))], 1)
    f, g = oracle_lib.overlap_grad(c, pi, pj, params)
    f_plain = oracle_lib.overlap(c, pi, pj, params=params)
    np.testing.assert_allclose(f, f_plain, rtol=1e-14, atol=0)
    h = 1e-5
    fd = np.empty_like(g)
    for k in range(3):
        pp, pm = params.copy(), params.copy()
        pp[:, k] += h
        pm[:, k] -= h
        fd[:, k] = (oracle_lib.overlap(c, pi, pj, params=pp)
                    - oracle_lib.overlap(c, pi, pj, params=pm)) / (2 * h)
    scale = np.abs(g).max(1, keepdims=True)
    assert np.all(np.abs(fd - g) <= 1e-7 * scale)


def test_gradient_single_points_closed_form(oracle_lib):
    # one point each, theta = 0: df/dt = e (xa - xb - t) / s2,
    # df/dtheta = e (d . J xb) / s2 with J xb = (-yb, xb)
    c = {"dim": 2, "offsets": np.array([0, 1, 2], np.int64),
         "x": np.array([0.1, 0.02], np.float32), "y": np.array([-0.03, 0.05], np.float32),
         "z": None, "sigma": np.array([0.07, 0.05], np.float32), "weight": None}
    t = np.array([0.01, -0.02])
    f, g = oracle_lib.overlap_grad(c, [0], [1], np.array([[0.0, t[0], t[1]]]))
    xa = np.array([c["x"][0], c["y"][0]], np.float64)
    xb = np.array([c["x"][1], c["y"][1]], np.float64)
    s2 = float(c["sigma"][0]) ** 2 + float(c["sigma"][1]) ** 2
    d = xa - xb - t
    e = np.exp(-(d @ d) / (2 * s2))
    assert abs(f[0] - e) <= 1e-15
    np.testing.assert_allclose(g[0, 1:], e * d / s2, rtol=1e-13)
    np.testing.assert_allclose(g[0, 0], e * (d @ np.array([-xb[1], xb[0]])) / s2, rtol=1e-13)


def test_conditioning_outputs(oracle_lib):
    c = synth.clouds_uniform(n=6, dim=2, size=(10, 20), seed=1)
    pi, pj = oracle_lib.all_pairs(6)
    f, kappa, bound = oracle_lib.overlap(c, pi, pj, with_cond=True)
    assert np.all(kappa >= 0) and np.all(bound >= 0)
    # bound >= 4 * 2^-23 * f by construction
    assert np.all(bound >= 4 * 2.0 ** -23 * f * (1 - 1e-12))


def test_ascent_step_increases_cost_near_alignment(oracle_lib):
    # two copies of one template: start 0.05 off the known relative pose;
    # small steps on log f must not decrease f
    c = synth.clouds_templates(n=16, seed=3)
    pairs = [(i, j) for i in range(16) for j in range(i + 1, 16)
             if c["template"][i] == c["template"][j]]
    pi = np.array([p[0] for p in pairs])
    pj = np.array([p[1] for p in pairs])
    # pose of j relative to i: x_i ~ R_i T + t_i, x_j ~ R_j T + t_j
    # => x_i ~ R_i R_j^T (x_j - t_j) + t_i = R(th_i - th_j) x_j + t'
    prm = np.zeros((len(pi), 3))
    for q, (i, j) in enumerate(pairs):
        th = c["theta"][i] - c["theta"][j]
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        prm[q, 0] = th + 0.05
        prm[q, 1:] = c["t"][i] - R @ c["t"][j] + 0.05
    f_prev = None
    for _ in range(5):
        prm, f, g, flag = oracle_lib.ascent_step(c, pi, pj, prm, eta=1e-4)
        assert not flag.any()
        if f_prev is not None:
            assert np.all(f >= f_prev * (1 - 1e-12))
        f_prev = f


def _single_point_pairs():
    """Three pairs of single weighted points (item 2q against item 2q + 1)
    whose Gaussian terms sit well below 1, so that a step scaled by grad f
    instead of grad f / f moves the parameters by a visibly different
    amount."""
    xa = np.array([[0.10, -0.03], [-0.20, 0.15], [0.05, 0.05]])
    xb = np.array([[0.02, 0.05], [-0.10, 0.02], [0.12, -0.04]])
    sa = np.array([0.07, 0.06, 0.05])
    sb = np.array([0.05, 0.08, 0.04])
    wa = np.array([2.0, 0.7, 1.3])
    wb = np.array([0.7, 1.9, 0.4])
    pts = np.empty((6, 2))
    pts[0::2], pts[1::2] = xa, xb
    sig = np.empty(6); sig[0::2], sig[1::2] = sa, sb
    w = np.empty(6); w[0::2], w[1::2] = wa, wb
    c = {"dim": 2, "offsets": np.arange(7, dtype=np.int64),
         "x": pts[:, 0].astype(np.float32), "y": pts[:, 1].astype(np.float32), "z": None,
         "sigma": sig.astype(np.float32), "weight": w.astype(np.float32)}
    params = np.array([[0.3, 0.01, -0.02], [-0.7, 0.05, 0.03], [1.1, -0.04, 0.06]])
    return c, np.array([0, 2, 4]), np.array([1, 3, 5]), params


def test_ascent_step_single_points_closed_form(oracle_lib):
    # One point per item: f = wa wb e, e = exp(-|d|^2 / (2 s^2)),
    # d = xa - (R(theta) xb + t), s^2 = sa^2 + sb^2.  Ascent on log f moves
    # (theta, t) by eta grad f / f = eta (d . R'(theta) xb, d) / s^2: the
    # weights and e cancel.  The values below are computed from the float32
    # inputs with numpy, independently of the oracle.
    c, pi, pj, p0 = _single_point_pairs()
    eta = 1e-2
    x = np.stack([c["x"], c["y"]], 1).astype(np.float64)
    s = c["sigma"].astype(np.float64)
    w = c["weight"].astype(np.float64)
    want = p0.copy()
    f_want = np.empty(3)
    for q, (a, b) in enumerate(zip(pi, pj)):
        th, t = p0[q, 0], p0[q, 1:]
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        dR = np.array([[-np.sin(th), -np.cos(th)], [np.cos(th), -np.sin(th)]])
        d = x[a] - (R @ x[b] + t)
        s2 = s[a] ** 2 + s[b] ** 2
        f_want[q] = w[a] * w[b] * np.exp(-(d @ d) / (2 * s2))
        want[q, 0] += eta * (d @ (dR @ x[b])) / s2
        want[q, 1:] += eta * d / s2
    assert np.all((f_want > 0.05) & (f_want < 0.95 * w[pi] * w[pj]))   # e well below 1
    got, f, g, flag = oracle_lib.ascent_step(c, pi, pj, p0, eta=eta)
    assert not flag.any()
    np.testing.assert_allclose(f, f_want, rtol=1e-13)
    np.testing.assert_allclose(got - p0, want - p0, rtol=1e-11, atol=0)
    # the step is eta grad f / f of the oracle's own (separately pinned) gradient
    np.testing.assert_allclose(got - p0, eta * g / f[:, None], rtol=1e-13, atol=0)


def test_ascent_step_skips_and_flags_below_fmin(oracle_lib):
    # pairs whose f falls below fmin keep their parameters and are flagged;
    # the others take their step as usual
    c, pi, pj, p0 = _single_point_pairs()
    f0, _ = oracle_lib.overlap_grad(c, pi, pj, p0)
    fmin = float(np.median(f0))                 # pair with the smallest f is skipped
    low = f0 < fmin
    assert low.sum() == 1
    got, f, g, flag = oracle_lib.ascent_step(c, pi, pj, p0, eta=1e-2, fmin=fmin)
    assert np.array_equal(flag.astype(bool), low)
    assert np.array_equal(got[low], p0[low])
    assert np.all(np.abs(got[~low] - p0[~low]).max(1) > 0)
    # every pair skipped when fmin exceeds all of them
    got, _, _, flag = oracle_lib.ascent_step(c, pi, pj, p0, eta=1e-2, fmin=10.0)
    assert flag.all() and np.array_equal(got, p0)


def test_ascent_step_goes_uphill_on_log_f(oracle_lib):
    # a small step must raise log f by about eta |grad log f|^2 (first order):
    # a sign error lowers f, a missing 1/f scales the gain by f
    c, pi, pj, p0 = _single_point_pairs()
    eta = 1e-6
    got, f, g, _ = oracle_lib.ascent_step(c, pi, pj, p0, eta=eta)
    f1, _ = oracle_lib.overlap_grad(c, pi, pj, got)
    gain = np.log(f1) - np.log(f)
    first_order = eta * ((g / f[:, None]) ** 2).sum(1)
    np.testing.assert_allclose(gain, first_order, rtol=1e-3)
