"""Pins for the oracle's cosine of sparse composition vectors (Sec. V-B).

The merge of two sorted index lists is held to the same cosine computed a
second way (rows scattered into dense FP64 vectors, numpy dot products and
norms), and to exact properties: self-cosine 1, symmetry, 0 on disjoint
supports, invariance to positive scaling and a sign flip for negative, NaN
for an empty row."""
import numpy as np

import synth


def _dense(off, idx, val, dim):
    n = len(off) - 1
    X = np.zeros((n, dim))
    for i in range(n):
        X[i, idx[off[i]:off[i + 1]]] = val[off[i]:off[i + 1]]
    return X


def test_cosine_matches_dense_form(oracle_lib):
    dim = 3000
    off, idx, val = synth.sparse_cv(12, dim=dim, nnz=(20, 900), common=300, seed=3)
    X = _dense(off, idx, val, dim)
    pi, pj = np.triu_indices(12, 1)
    ref = (X[pi] * X[pj]).sum(1) / np.sqrt((X[pi] ** 2).sum(1) * (X[pj] ** 2).sum(1))
    np.testing.assert_allclose(oracle_lib.sparse_cosine(off, idx, val, pi, pj), ref,
                               rtol=1e-12, atol=1e-14)


def test_cosine_exact_properties(oracle_lib):
    dim = 2000
    off, idx, val = synth.sparse_cv(8, dim=dim, nnz=(10, 500), common=200, seed=4)
    ii = np.arange(8)
    np.testing.assert_allclose(oracle_lib.sparse_cosine(off, idx, val, ii, ii), 1.0, atol=1e-14)
    pi, pj = np.triu_indices(8, 1)
    c = oracle_lib.sparse_cosine(off, idx, val, pi, pj)
    np.testing.assert_array_equal(oracle_lib.sparse_cosine(off, idx, val, pj, pi), c)
    assert np.all(np.abs(c) <= 1.0)
    # positive scaling of one row changes nothing; a negative one flips the sign
    v2 = val.copy()
    v2[off[2]:off[3]] *= 4.0                                # exact in FP32
    v2[off[5]:off[6]] *= -1.0
    c2 = oracle_lib.sparse_cosine(off, idx, v2, pi, pj)
    flip = (pi == 5) | (pj == 5)
    np.testing.assert_allclose(c2[~flip], c[~flip], rtol=1e-12)
    np.testing.assert_allclose(c2[flip], -c[flip], rtol=1e-12)


def test_cosine_disjoint_and_empty(oracle_lib):
    off = np.array([0, 3, 6, 6], np.int64)
    idx = np.array([1, 5, 9, 2, 6, 10], np.int32)          # rows 0, 1 disjoint; row 2 empty
    val = np.array([1.0, -2.0, 0.5, 3.0, 1.0, -1.0], np.float32)
    c = oracle_lib.sparse_cosine(off, idx, val, [0, 0, 1], [1, 2, 2])
    assert c[0] == 0.0 and np.isnan(c[1]) and np.isnan(c[2])
    # one shared code: the cosine is the product over the norms
    idx2 = idx.copy()
    idx2[3] = 5
    idx2[3:6] = np.sort(idx2[3:6])
    c = oracle_lib.sparse_cosine(off, idx2, val, [0], [1])
    shared = -2.0 * 3.0
    np.testing.assert_allclose(c[0], shared / np.sqrt((1 + 4 + 0.25) * (9 + 1 + 1)), rtol=1e-12)
