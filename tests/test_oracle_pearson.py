"""Pins for the oracle's Pearson correlation and per-item statistics.

Pinned to: the one-pass textbook formula in extended precision, self
correlation 1, exact symmetry, the [-1, 1] range, invariance under an exact
affine change of units, numpy's own mean/variance, and the correlation the
input noise model implies for items of one group.
"""
import numpy as np
import pytest

import synth


def _grid_vectors(rng, n, D):
    # values k * 2^-8, |k| < 2^10: exact under x -> 2x + 1 in FP32
    return (rng.integers(-1000, 1000, size=(n, D)) * 2.0 ** -8).astype(np.float32)


@pytest.mark.parametrize("D", [2, 5, 16])
def test_pearson_matches_one_pass_long_double(oracle_lib, D):
    rng = np.random.default_rng(D)
    X = rng.standard_normal((6, D)).astype(np.float32)
    pi, pj = oracle_lib.all_pairs(6)
    r = oracle_lib.pearson(X, pi, pj, n_threads=2)
    L = X.astype(np.longdouble)
    ref = []
    for i, j in zip(pi, pj):
        xi, xj = L[i], L[j]
        mi, mj = xi.sum() / D, xj.sum() / D
        sxy = (xi * xj).sum() - D * mi * mj
        sxx = (xi * xi).sum() - D * mi * mi
        syy = (xj * xj).sum() - D * mj * mj
        ref.append(float(sxy / np.sqrt(sxx * syy)))
    np.testing.assert_allclose(r, ref, rtol=0, atol=1e-12)


def test_stats_match_numpy(oracle_lib):
    rng = np.random.default_rng(1)
    X = (3.0 + rng.standard_normal((5, 1000))).astype(np.float32)
    mu, ss = oracle_lib.vector_stats(X)
    X64 = X.astype(np.float64)
    np.testing.assert_allclose(mu, X64.mean(1), rtol=1e-14)
    np.testing.assert_allclose(ss, X64.var(1) * X.shape[1], rtol=1e-12)


def test_self_correlation_symmetry_range(oracle_lib):
    rng = np.random.default_rng(2)
    X = rng.standard_normal((9, 4096)).astype(np.float32)
    idx = np.arange(9)
    r_self = oracle_lib.pearson(X, idx, idx)
    assert np.all(np.abs(r_self - 1.0) <= 1e-14)
    pi, pj = oracle_lib.all_pairs(9)
    r1 = oracle_lib.pearson(X, pi, pj)
    r2 = oracle_lib.pearson(X, pj, pi)
    assert np.array_equal(r1, r2)
    assert np.all(np.abs(r1) <= 1.0)


def test_affine_invariance(oracle_lib):
    rng = np.random.default_rng(3)
    X = _grid_vectors(rng, 5, 777)
    Y = (2.0 * X + 1.0).astype(np.float32)
    assert np.array_equal((Y - 1.0) / 2.0, X)        # the change of units is exact
    pi, pj = oracle_lib.all_pairs(5)
    np.testing.assert_allclose(oracle_lib.pearson(Y, pi, pj), oracle_lib.pearson(X, pi, pj),
                               rtol=0, atol=1e-14)


def test_kahan_bounds_plain_sum(oracle_lib):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((4, 1 << 16)).astype(np.float32)
    pi, pj = oracle_lib.all_pairs(4)
    a = oracle_lib.pearson(X, pi, pj)
    b = oracle_lib.pearson(X, pi, pj, kahan=True)
    assert np.max(np.abs(a - b)) < 1e-13


def test_noise_model_group_correlation(oracle_lib):
    # x = eps + 0.05 g_group: within a group r ~ 0.05^2 / (1 + 0.05^2) = 0.002494,
    # across groups r ~ 0, spread ~ 1 / sqrt(D)
    n, D = 256, 1 << 16
    X = synth.vectors_grouped(n, D, seed=5).numpy()
    gid = synth.group_ids(n, 16, seed=5)
    assert np.all(np.bincount(gid) == 16)
    pi, pj = oracle_lib.all_pairs(n)
    r = oracle_lib.pearson(X, pi, pj)
    same = gid[pi] == gid[pj]
    expect = 0.05 ** 2 / (1 + 0.05 ** 2)
    assert abs(r[same].mean() - expect) < 5e-4
    assert abs(r[~same].mean()) < 2e-4
    assert abs(r[~same].std() * np.sqrt(D) - 1.0) < 0.05
