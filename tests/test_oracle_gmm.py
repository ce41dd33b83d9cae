"""Pins for the oracle's particle scores: the squared L2 distance between
Gaussian mixtures and the Bhattacharyya cost (Sec. V-C names both).

Each pin holds the oracle to something other than itself: grid quadrature of
the defining integrals (the squared difference of two weighted normal
densities, the square root of their product), the factorisation of a 3-D
isotropic Gaussian into three 1-D ones, mixtures as sums of single-component
items, explicitly moved coordinates for the transform, and exact properties
of a distance (zero on the diagonal, non-negative, symmetric, rigid
invariance).
"""
import numpy as np
import pytest


def _cloud(points, sigma, weight, dim):
    """Items given as lists of (points [k, dim], sigma [k], weight [k])."""
    off = np.zeros(len(points) + 1, np.int64)
    np.cumsum([len(p) for p in points], out=off[1:])
    P = np.concatenate(points).astype(np.float64)
    return {"dim": dim, "offsets": off,
            "x": P[:, 0].astype(np.float32), "y": P[:, 1].astype(np.float32),
            "z": P[:, 2].astype(np.float32) if dim == 3 else None,
            "sigma": np.concatenate(sigma).astype(np.float32),
            "weight": np.concatenate(weight).astype(np.float32)}


def _random_clouds(rng, n, dim, max_pts=5):
    pts, sg, wt = [], [], []
    for _ in range(n):
        k = int(rng.integers(1, max_pts + 1))
        pts.append(rng.uniform(-0.3, 0.3, size=(k, dim)))
        sg.append(rng.uniform(0.05, 0.15, size=k))
        wt.append(rng.uniform(0.5, 2.0, size=k))
    return _cloud(pts, sg, wt, dim)


def _normal2(X, Y, m, s):
    return np.exp(-((X - m[0]) ** 2 + (Y - m[1]) ** 2) / (2 * s * s)) / (2 * np.pi * s * s)


def _normal1(x, m, s):
    return np.exp(-(x - m) ** 2 / (2 * s * s)) / np.sqrt(2 * np.pi * s * s)


def _single_pair(a, b, sa, sb, wa, wb, dim):
    f32 = lambda v: np.float32(v).astype(np.float64)
    a, b = np.array([f32(v) for v in a]), np.array([f32(v) for v in b])
    return _cloud([a[None, :], b[None, :]], [[sa], [sb]], [[wa], [wb]], dim), a, b


@pytest.mark.parametrize("case", range(4))
def test_single_components_match_quadrature_2d(oracle_lib, case):
    rng = np.random.default_rng(100 + case)
    sa, sb = (float(np.float32(v)) for v in rng.uniform(0.05, 0.12, 2))
    wa, wb = (float(np.float32(v)) for v in rng.uniform(0.5, 2.0, 2))
    c, a, b = _single_pair(rng.uniform(-0.1, 0.1, 2), rng.uniform(-0.1, 0.1, 2), sa, sb, wa, wb, 2)
    h = 0.0015
    g = np.arange(-0.9, 0.9 + h / 2, h)
    X, Y = np.meshgrid(g, g, indexing="ij")
    p = wa * _normal2(X, Y, a, sa)
    q = wb * _normal2(X, Y, b, sb)
    l2 = ((p - q) ** 2).sum() * h * h
    bc = np.sqrt(p * q).sum() * h * h
    got_l2 = oracle_lib.gmm_l2(c, [0], [1])[0]
    got_bc = oracle_lib.bhattacharyya(c, [0], [1])[0]
    S = oracle_lib.gmm_self(c)
    np.testing.assert_allclose(got_l2, l2, rtol=1e-6)
    np.testing.assert_allclose(got_bc, bc, rtol=1e-6)
    np.testing.assert_allclose(S, [(p * p).sum() * h * h, (q * q).sum() * h * h], rtol=1e-6)


def test_single_components_3d_factorise(oracle_lib):
    """A 3-D isotropic Gaussian is the product of three 1-D ones, so the
    cross integral and the Bhattacharyya coefficient are products of 1-D
    quadratures."""
    rng = np.random.default_rng(7)
    sa, sb = (float(np.float32(v)) for v in rng.uniform(0.05, 0.12, 2))
    c, a, b = _single_pair(rng.uniform(-0.1, 0.1, 3), rng.uniform(-0.1, 0.1, 3), sa, sb, 1.0, 1.0, 3)
    h = 1e-4
    x = np.arange(-1.0, 1.0 + h / 2, h)
    cross, bc = 1.0, 1.0
    for k in range(3):
        pa, pb = _normal1(x, a[k], sa), _normal1(x, b[k], sb)
        cross *= (pa * pb).sum() * h
        bc *= np.sqrt(pa * pb).sum() * h
    self_a = (_normal1(x, 0.0, sa) ** 2).sum() * h
    self_b = (_normal1(x, 0.0, sb) ** 2).sum() * h
    l2 = self_a ** 3 + self_b ** 3 - 2 * cross
    np.testing.assert_allclose(oracle_lib.gmm_l2(c, [0], [1])[0], l2, rtol=1e-8)
    np.testing.assert_allclose(oracle_lib.bhattacharyya(c, [0], [1])[0], bc, rtol=1e-8)


@pytest.mark.parametrize("dim", [2, 3])
def test_mixtures_are_sums_of_components(oracle_lib, dim):
    """Cross and Bhattacharyya terms of two mixtures = the sum of their
    single-component pairs (each item split into one item per point)."""
    rng = np.random.default_rng(dim)
    c = _random_clouds(rng, 2, dim, max_pts=4)
    off = c["offsets"]
    pts = np.stack([c[k] for k in (["x", "y", "z"] if dim == 3 else ["x", "y"])], 1)
    singles = _cloud([pts[k:k + 1] for k in range(off[-1])], [c["sigma"][k:k + 1] for k in range(off[-1])],
                     [c["weight"][k:k + 1] for k in range(off[-1])], dim)
    A, B = range(off[0], off[1]), range(off[1], off[2])
    pi = np.array([a for a in A for b in B]); pj = np.array([b for a in A for b in B])
    bc_parts = oracle_lib.bhattacharyya(singles, pi, pj)
    np.testing.assert_allclose(oracle_lib.bhattacharyya(c, [0], [1])[0], bc_parts.sum(), rtol=1e-12)
    # cross term from the distance: C = (S_i + S_j - d) / 2, against the
    # single-component distances of every point pair
    S = oracle_lib.gmm_self(c)
    C = (S[0] + S[1] - oracle_lib.gmm_l2(c, [0], [1])[0]) / 2
    Ss = oracle_lib.gmm_self(singles)
    C_parts = (Ss[pi] + Ss[pj] - oracle_lib.gmm_l2(singles, pi, pj)) / 2
    np.testing.assert_allclose(C, C_parts.sum(), rtol=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_distance_properties(oracle_lib, dim):
    rng = np.random.default_rng(30 + dim)
    c = _random_clouds(rng, 8, dim)
    n = 8
    ii = np.arange(n)
    S = oracle_lib.gmm_self(c)
    d_diag = oracle_lib.gmm_l2(c, ii, ii)
    assert np.all(np.abs(d_diag) <= 1e-12 * S)
    pi, pj = np.triu_indices(n, 1)
    d = oracle_lib.gmm_l2(c, pi, pj)
    assert np.all(d > 0)                                   # a squared norm of p_i - p_j != 0
    np.testing.assert_allclose(oracle_lib.gmm_l2(c, pj, pi), d, rtol=1e-12)
    f = oracle_lib.bhattacharyya(c, pi, pj)
    np.testing.assert_allclose(oracle_lib.bhattacharyya(c, pj, pi), f, rtol=1e-12)
    # a lone component against itself: coefficient 1, times sqrt(w w) = w
    single = _cloud([np.zeros((1, dim))], [[0.07]], [[1.7]], dim)
    np.testing.assert_allclose(oracle_lib.bhattacharyya(single, [0], [0])[0], np.float32(1.7), rtol=1e-6)


def test_rigid_invariance_and_transform(oracle_lib):
    """Moving both items by one rigid motion changes nothing; a transform
    parameter equals moving the second item's points explicitly."""
    rng = np.random.default_rng(5)
    c = _random_clouds(rng, 2, 2)
    th, tx, ty = 0.4, 0.05, -0.03
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    P = np.stack([c["x"], c["y"]], 1).astype(np.float64)
    moved = dict(c)
    Q = P @ R.T + np.array([tx, ty])
    moved["x"], moved["y"] = Q[:, 0].astype(np.float32), Q[:, 1].astype(np.float32)
    for fn in (oracle_lib.gmm_l2, oracle_lib.bhattacharyya):
        np.testing.assert_allclose(fn(moved, [0], [1]), fn(c, [0], [1]), rtol=1e-5)
    # the transform acts on item j: compare with item j's points moved by hand
    j_moved = dict(c)
    sl = slice(c["offsets"][1], c["offsets"][2])
    Q = P.copy()
    Q[sl] = P[sl] @ R.T + np.array([tx, ty])
    j_moved["x"], j_moved["y"] = Q[:, 0].astype(np.float32), Q[:, 1].astype(np.float32)
    prm = np.array([[th, tx, ty]])
    for fn in (oracle_lib.gmm_l2, oracle_lib.bhattacharyya):
        np.testing.assert_allclose(fn(c, [0], [1], params=prm), fn(j_moved, [0], [1]), rtol=1e-5)
