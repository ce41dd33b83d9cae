"""Pins for the oracle's pair indexing and divide-and-conquer order.

Pinned to: the pair counts printed in Table I (tests/golden), brute-force
enumeration of the strict upper triangle, and Morton (Z) order for the
recursive quadrant split of Sec. IV-B on power-of-two sizes.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_pair_counts.txt")


def _golden_counts():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            n, p = line.split()
            rows.append((int(n), int(p)))
    return rows


def test_pair_count_matches_paper_table(oracle_lib):
    rows = _golden_counts()
    assert len(rows) == 2
    for n, p in rows:
        assert oracle_lib.pair_count(n) == p


@pytest.mark.parametrize("n", [0, 1, 2, 3, 7, 16, 33])
def test_pair_count_brute_force(oracle_lib, n):
    brute = sum(1 for i in range(n) for j in range(n) if i < j)
    assert oracle_lib.pair_count(n) == brute


@pytest.mark.parametrize("n", [2, 5, 17, 40])
def test_pair_index_is_row_major_enumeration(oracle_lib, n):
    k = 0
    for i in range(n):
        for j in range(i + 1, n):
            assert oracle_lib.pair_index(i, j, n) == k
            k += 1
    assert k == oracle_lib.pair_count(n)
    # out-of-range and lower-triangle entries have no index
    assert oracle_lib.pair_index(1, 1, n) == -1
    assert oracle_lib.pair_index(1, 0, n) == -1
    assert oracle_lib.pair_index(0, n, n) == -1


@pytest.mark.parametrize("n", [2, 3, 8, 13, 64, 100])
def test_dc_order_covers_each_pair_once(oracle_lib, n):
    oi, oj = oracle_lib.dc_order(n)
    assert len(oi) == n * (n - 1) // 2
    assert np.all(oi < oj) and np.all(oi >= 0) and np.all(oj < n)
    keys = oi * n + oj
    assert len(np.unique(keys)) == len(keys)


def _morton_key(i, j, bits):
    # row bit above column bit at every level: quadrants TL, TR, BL, BR
    k = 0
    for b in range(bits - 1, -1, -1):
        k = (k << 2) | (((i >> b) & 1) << 1) | ((j >> b) & 1)
    return k


@pytest.mark.parametrize("n", [8, 32])
def test_dc_order_is_quadrant_z_order(oracle_lib, n):
    bits = int(np.log2(n))
    oi, oj = oracle_lib.dc_order(n)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    pairs.sort(key=lambda p: _morton_key(p[0], p[1], bits))
    assert list(zip(oi.tolist(), oj.tolist())) == pairs


def test_dc_order_quadrants_are_contiguous(oracle_lib):
    # every aligned sub-quadrant at every level occupies one contiguous run
    n = 16
    oi, oj = oracle_lib.dc_order(n)
    for size in (8, 4, 2):
        for r0 in range(0, n, size):
            for c0 in range(0, n, size):
                sel = np.nonzero((oi // size == r0 // size) & (oj // size == c0 // size))[0]
                if len(sel):
                    assert sel[-1] - sel[0] + 1 == len(sel)
