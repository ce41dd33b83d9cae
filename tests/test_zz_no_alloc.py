"""The allocation-free Pearson entry point (ap_pearson_fp32_noalloc).

It serves callers that must not let the library allocate GPU memory, for
example processes whose device memory is owned by their own pool allocator,
or services with a hard cap on what one request may allocate.  Checked here
through the C ABI against the FP64 oracle element by element and against the
library's regular FP32 path, on two calls in a row, plus its size limit and
that a call leaves the device's free memory unchanged.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import pearson_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import paper_2009_04755_gb300 as ap
    L = ap.lib()
    fn = L.ap_pearson_fp32_noalloc
    fn.restype = ctypes.c_int32
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.c_void_p]
    return ap, fn


def _noalloc(fn, X, out):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], X.stride(0),
              ctypes.c_void_p(out.data_ptr()), s)


def _regular(ap, X):
    with ap.Items.from_vectors(X, precisions=(ap.AP_PREC_FP32,)) as it:
        return it.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32).cpu().numpy()


def test_noalloc_matches_oracle_and_regular_fp32_path_twice(lib, oracle_lib):
    ap, fn = lib
    n, D = 300, 1500
    pi, pj = np.triu_indices(n, 1)
    for seed in (21, 22):                       # two calls in a row, different data
        Xh = synth.vectors_grouped(n, D, seed=seed)
        X = Xh.cuda()
        out = torch.full((n * (n - 1) // 2,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(fn, X, out) == ap.binding.AP_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        tol = pearson_tolerance(Xh.numpy(), pi, pj, ap.AP_PREC_FP32)
        assert np.all(np.isfinite(got))
        # the FP64 oracle on every pair, element by element
        ref = oracle_lib.pearson(Xh.numpy(), pi, pj)
        assert np.all(np.abs(got - ref) <= tol), float(np.abs(got - ref).max())
        # and the library's regular FP32 path on the same rows
        want = _regular(ap, X)
        assert np.all(np.abs(got - want) <= tol), float(np.abs(got - want).max())


def test_noalloc_ragged_rows_and_stride(lib, oracle_lib):
    ap, fn = lib
    n, D, ld = 131, 77, 80                      # ragged tiles, unaligned row stride
    base = torch.randn(n, ld, device="cuda")
    X = base[:, :D]
    out = torch.empty(n * (n - 1) // 2, dtype=torch.float64, device="cuda")
    assert _noalloc(fn, X, out) == ap.binding.AP_OK
    torch.cuda.synchronize()
    want = _regular(ap, X.contiguous())
    pi, pj = np.triu_indices(n, 1)
    tol = pearson_tolerance(X.cpu().numpy(), pi, pj, ap.AP_PREC_FP32)
    assert np.all(np.abs(out.cpu().numpy() - want) <= tol)
    ref = oracle_lib.pearson(X.cpu().numpy(), pi, pj)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= tol)


def test_noalloc_allocates_nothing_and_rejects_oversize(lib):
    ap, fn = lib
    n, D = 257, 512
    X = torch.randn(n, D, device="cuda")
    out = torch.empty(n * (n - 1) // 2, dtype=torch.float64, device="cuda")
    assert _noalloc(fn, X, out) == ap.binding.AP_OK       # first call sets up the device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(fn, X, out) == ap.binding.AP_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # beyond the scratch array's capacity: rejected before any device work
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    too_many = 65536 + 1
    assert fn(ctypes.c_void_p(X.data_ptr()), too_many, D, D, ctypes.c_void_p(out.data_ptr()),
              s) == ap.binding.AP_ERR_UNSUPPORTED
    assert fn(None, n, D, D, ctypes.c_void_p(out.data_ptr()), s) == ap.binding.AP_ERR_INVALID_ARG
    assert fn(ctypes.c_void_p(X.data_ptr()), n, 1, 1, ctypes.c_void_p(out.data_ptr()),
              s) == ap.binding.AP_ERR_INVALID_ARG
