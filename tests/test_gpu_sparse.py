"""GPU parity of the sparse composition-vector cosine (Sec. V-B) against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ap():
    import paper_2009_04755_gb300 as ap
    ap.lib()
    return ap


def _tolerance(oracle_lib, off, idx, val, pi, pj):
    """FP32 products (relative error 2^-24 each) summed in FP32 per lane over
    at most 64 chunks before FP64 (at most 2^-24 x 64 of the partial sums'
    magnitudes): |err| <= 2^-17 sum_k |a_ik a_jk| / sqrt(ss_i ss_j), which is
    2^-17 times the cosine of the absolute values."""
    mag = oracle_lib.sparse_cosine(off, idx, np.abs(val), pi, pj)
    return 2.0 ** -17 * np.nan_to_num(mag) + 1e-12


def _check(ap, oracle_lib, off, idx, val, dim, device_input=False):
    n = len(off) - 1
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.sparse_cosine(off, idx, val, pi, pj)
    if device_input:
        it = ap.Items.from_sparse(off, torch.from_numpy(idx).cuda(), torch.from_numpy(val).cuda(), dim)
    else:
        it = ap.Items.from_sparse(off, idx, val, dim)
    with it:
        got = it.run_pairs(ap.AP_FN_COSINE).cpu().numpy()
        cnt = it.run_pairs(ap.AP_FN_COVERAGE).cpu().numpy()
        assert it.last_device_error() == 0
    assert np.all(cnt == 1)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    tol = _tolerance(oracle_lib, off, idx, val, pi, pj)
    err = np.abs(got[~nan] - ref[~nan])
    assert np.all(err <= tol[~nan]), float((err / tol[~nan]).max())
    return got


@pytest.mark.parametrize("n,dim,nnz", [(70, 20000, (5, 3000)), (33, 2048, (1, 2048)),
                                       (2, 5000, (100, 4000)), (300, 160000, (1000, 20000))])
def test_cosine_all_pairs(ap, oracle_lib, n, dim, nnz):
    off, idx, val = synth.sparse_cv(n, dim=dim, nnz=nnz, common=min(dim, 1500), seed=n)
    _check(ap, oracle_lib, off, idx, val, dim)


def test_cosine_device_input_and_edges(ap, oracle_lib):
    """Device-resident CSR; empty rows (NaN), a row of zero values (NaN),
    codes on chunk boundaries, one-code rows, a dim that is not a multiple of
    the chunk."""
    dim = 3 * 2048 + 77
    rows = [np.array([], np.int64), np.array([0, 2047, 2048, 4095, 4096, dim - 1]),
            np.array([2047, 2048]), np.arange(0, dim, 3), np.array([5]), np.array([5]),
            np.arange(2040, 2060), np.array([dim - 1]), np.arange(100, 6000, 7)]
    rng = np.random.default_rng(1)
    off = np.zeros(len(rows) + 1, np.int64)
    np.cumsum([len(r) for r in rows], out=off[1:])
    idx = np.concatenate(rows).astype(np.int32)
    val = rng.standard_normal(len(idx)).astype(np.float32)
    val[off[7]:off[8]] = 0.0                                   # a row of zeros
    _check(ap, oracle_lib, off, idx, val, dim, device_input=True)


def test_cosine_rejects_bad_rows(ap):
    off = np.array([0, 3, 5], np.int64)
    with pytest.raises(ap.APError):                            # not increasing
        ap.Items.from_sparse(off, np.array([1, 5, 4, 0, 2], np.int32),
                             np.ones(5, np.float32), 100)
    with pytest.raises(ap.APError):                            # code >= dim
        ap.Items.from_sparse(off, np.array([1, 5, 9, 0, 100], np.int32),
                             np.ones(5, np.float32), 100)
    with pytest.raises(ap.APError):                            # duplicate code
        ap.Items.from_sparse(off, np.array([1, 5, 5, 0, 2], np.int32),
                             np.ones(5, np.float32), 100)
