"""FP64 CPU oracle for the all-pairs method -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The product path (the CUDA library and its binding)
never does, and this package never imports the product.

The arithmetic lives in ``oracle.c`` (plain C, double precision, double loops);
this module only compiles it with gcc and marshals numpy arrays through ctypes.
Every function cites the passage of the paper it follows:

* ``pair_count`` / ``pair_index`` -- the problem statement f(l(i), l(j)) for
  every i < j (Sec. III) and the n(n-1)/2 pair count (Sec. VI-A).
* ``dc_order`` -- recursive quadrant splitting of the upper triangle, empty
  quadrants skipped (Sec. IV-B).
* ``overlap`` / ``overlap_grad`` / ``ascent_step`` -- the Gaussian overlap
  cost between weighted point clouds, the cross term of the GMM L2 distance
  of the microscopy application (Sec. V-C), and its analytic adjoint with
  respect to (theta, tx, ty).
* ``vector_stats`` / ``pearson`` -- normalised cross correlation of dense
  vectors (forensics application, Sec. V-A), two-pass centred sums.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, no fast-math)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            vp = ctypes.c_void_p
            lib.or_pair_count.restype = i64
            lib.or_pair_count.argtypes = [i64]
            lib.or_pair_index.restype = i64
            lib.or_pair_index.argtypes = [i64, i64, i64]
            lib.or_dc_order.restype = i64
            lib.or_dc_order.argtypes = [i64, vp, vp]
            lib.or_overlap_pairs.restype = None
            lib.or_overlap_pairs.argtypes = [i32, vp, vp, vp, vp, vp, vp, i64, vp, vp,
                                             vp, vp, vp, vp, i32]
            lib.or_gmm_pairs.restype = None
            lib.or_gmm_pairs.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp,
                                         vp, vp, i32]
            lib.or_gmm_self.restype = None
            lib.or_gmm_self.argtypes = [i32, vp, vp, vp, vp, vp, vp, i64, vp, vp, i32]
            lib.or_sparse_cosine_pairs.restype = None
            lib.or_sparse_cosine_pairs.argtypes = [vp, vp, vp, i64, vp, vp, vp, i32]
            lib.or_overlap_grad_pairs.restype = None
            lib.or_overlap_grad_pairs.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp,
                                                  vp, vp, i32]
            lib.or_vector_stats.restype = None
            lib.or_vector_stats.argtypes = [i64, i64, i64, vp, vp, vp, i32]
            lib.or_pearson_pairs.restype = None
            lib.or_pearson_pairs.argtypes = [i64, i64, vp, vp, vp, i64, vp, vp, i32,
                                             vp, i32]
            lib.or_ascent_step.restype = None
            lib.or_ascent_step.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp, dbl, dbl,
                                           vp, vp, vp, i32]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def pair_count(n: int) -> int:
    """n(n-1)/2 unordered pairs (Sec. VI-A)."""
    return int(_load().or_pair_count(int(n)))


def pair_index(i: int, j: int, n: int) -> int:
    """Row-major packed index of pair (i, j), i < j (Sec. III)."""
    return int(_load().or_pair_index(int(i), int(j), int(n)))


def all_pairs(n: int):
    """Every (i, j) with 0 <= i < j < n in packed (row-major) order."""
    i, j = np.triu_indices(n, k=1)
    return i.astype(np.int64), j.astype(np.int64)


def dc_order(n: int):
    """Leaves of the recursive quadrant split of the upper triangle (Sec. IV-B)."""
    P = pair_count(n)
    oi = np.empty(max(P, 1), np.int64)
    oj = np.empty(max(P, 1), np.int64)
    k = _load().or_dc_order(int(n), _p(oi), _p(oj))
    return oi[:k], oj[:k]


def overlap(clouds: dict, pi, pj, params=None, n_threads: int | None = None,
            with_cond: bool = False):
    """Gaussian overlap cost f(i, j; theta, t) per listed pair, FP64 (Sec. V-C).

    ``clouds`` holds ``dim``, ``offsets`` (int64 [n+1]) and SoA float arrays
    ``x``, ``y``, ``z`` (3-D only), ``sigma``, ``weight`` (None = all ones).
    ``params`` is None (identity) or float [P, 3] = (theta, tx, ty).
    Returns f, or (f, kappa, bound) with ``with_cond``.
    """
    pi, pj = _i64(pi), _i64(pj)
    n = len(pi)
    f = np.empty(n, np.float64)
    kappa = np.empty(n, np.float64) if with_cond else None
    bound = np.empty(n, np.float64) if with_cond else None
    prm = None if params is None else np.ascontiguousarray(params, np.float64).reshape(-1)
    off = _i64(clouds["offsets"])
    x, y = _f32(clouds["x"]), _f32(clouds["y"])
    z = _f32(clouds.get("z")) if clouds["dim"] == 3 else None
    s, w = _f32(clouds["sigma"]), _f32(clouds.get("weight"))
    _load().or_overlap_pairs(int(clouds["dim"]), _p(off), _p(x), _p(y), _p(z), _p(s),
                             _p(w), n, _p(pi), _p(pj), _p(prm), _p(f), _p(kappa),
                             _p(bound), n_threads or default_threads())
    if with_cond:
        return f, kappa, bound
    return f


def _cloud_args(clouds):
    off = _i64(clouds["offsets"])
    x, y = _f32(clouds["x"]), _f32(clouds["y"])
    z = _f32(clouds.get("z")) if clouds["dim"] == 3 else None
    return off, x, y, z, _f32(clouds["sigma"]), _f32(clouds.get("weight"))


def _gmm(which, clouds, pi, pj, params, n_threads, with_bound):
    pi, pj = _i64(pi), _i64(pj)
    n = len(pi)
    out = np.empty(n, np.float64)
    bound = np.empty(n, np.float64) if with_bound else None
    prm = None if params is None else np.ascontiguousarray(params, np.float64).reshape(-1)
    off, x, y, z, s, w = _cloud_args(clouds)
    _load().or_gmm_pairs(which, int(clouds["dim"]), _p(off), _p(x), _p(y), _p(z), _p(s), _p(w),
                         n, _p(pi), _p(pj), _p(prm), _p(out), _p(bound),
                         n_threads or default_threads())
    return (out, bound) if with_bound else out


def gmm_l2(clouds: dict, pi, pj, params=None, n_threads: int | None = None,
           with_bound: bool = False):
    """Squared L2 distance S_i + S_j - 2 C_ij between the items as Gaussian
    mixtures (Sec. V-C's first particle score), FP64; pairs may have i == j."""
    return _gmm(1, clouds, pi, pj, params, n_threads, with_bound)


def bhattacharyya(clouds: dict, pi, pj, params=None, n_threads: int | None = None,
                  with_bound: bool = False):
    """Bhattacharyya cost sum_ab sqrt(w_a w_b) BC(N_a, N_b) (Sec. V-C's
    second particle score), FP64."""
    return _gmm(2, clouds, pi, pj, params, n_threads, with_bound)


def gmm_self(clouds: dict, n_threads: int | None = None, with_bound: bool = False):
    """S_i = integral of p_i^2 for every item, FP64."""
    off, x, y, z, s, w = _cloud_args(clouds)
    n = len(off) - 1
    S = np.empty(n, np.float64)
    bound = np.empty(n, np.float64) if with_bound else None
    _load().or_gmm_self(int(clouds["dim"]), _p(off), _p(x), _p(y), _p(z), _p(s), _p(w), n,
                        _p(S), _p(bound), n_threads or default_threads())
    return (S, bound) if with_bound else S


def sparse_cosine(off, idx, val, pi, pj, n_threads: int | None = None):
    """Cosine of sparse rows (CSR: off int64 [n+1], idx int32 sorted per row,
    val float32) per listed pair, FP64, by merging the index lists."""
    pi, pj = _i64(pi), _i64(pj)
    c = np.empty(len(pi), np.float64)
    off = _i64(off)
    idx = np.ascontiguousarray(idx, np.int32)
    val = _f32(val)
    _load().or_sparse_cosine_pairs(_p(off), _p(idx), _p(val), len(pi), _p(pi), _p(pj), _p(c),
                                   n_threads or default_threads())
    return c


def overlap_grad(clouds: dict, pi, pj, params=None, n_threads: int | None = None):
    """(f, g[P,3]) with g = df/d(theta, tx, ty), 2-D clouds, FP64."""
    assert clouds["dim"] == 2
    pi, pj = _i64(pi), _i64(pj)
    n = len(pi)
    f = np.empty(n, np.float64)
    g = np.empty((n, 3), np.float64)
    prm = None if params is None else np.ascontiguousarray(params, np.float64).reshape(-1)
    off = _i64(clouds["offsets"])
    x, y, s, w = (_f32(clouds["x"]), _f32(clouds["y"]), _f32(clouds["sigma"]),
                  _f32(clouds.get("weight")))
    _load().or_overlap_grad_pairs(_p(off), _p(x), _p(y), _p(s), _p(w), n, _p(pi), _p(pj),
                                  _p(prm), _p(f), _p(g), n_threads or default_threads())
    return f, g


def ascent_step(clouds: dict, pi, pj, params, eta: float, fmin: float = 1e-30,
                n_threads: int | None = None):
    """One ascent step p <- p + eta grad f / f per pair; returns (new_params, f, g, flag)."""
    pi, pj = _i64(pi), _i64(pj)
    n = len(pi)
    prm = np.array(params, np.float64, copy=True).reshape(n, 3)
    f = np.empty(n, np.float64)
    g = np.empty((n, 3), np.float64)
    flag = np.zeros(n, np.int32)
    off = _i64(clouds["offsets"])
    x, y, s, w = (_f32(clouds["x"]), _f32(clouds["y"]), _f32(clouds["sigma"]),
                  _f32(clouds.get("weight")))
    _load().or_ascent_step(_p(off), _p(x), _p(y), _p(s), _p(w), n, _p(pi), _p(pj),
                           _p(prm), float(eta), float(fmin), _p(f), _p(g), _p(flag),
                           n_threads or default_threads())
    return prm, f, g, flag


def vector_stats(X, n_threads: int | None = None):
    """(mu, ss) per row, two-pass FP64 (Sec. V-A pre-processing of the NCC)."""
    X = np.ascontiguousarray(X, np.float32)
    n, D = X.shape
    mu = np.empty(n, np.float64)
    ss = np.empty(n, np.float64)
    _load().or_vector_stats(n, D, D, _p(X), _p(mu), _p(ss), n_threads or default_threads())
    return mu, ss


def pearson(X, pi, pj, mu=None, ss=None, kahan: bool = False,
            n_threads: int | None = None):
    """Pearson r for the listed row pairs of X [n, D] (Sec. V-A), FP64."""
    X = np.ascontiguousarray(X, np.float32)
    n, D = X.shape
    if mu is None or ss is None:
        mu, ss = vector_stats(X, n_threads)
    mu = np.ascontiguousarray(mu, np.float64)
    ss = np.ascontiguousarray(ss, np.float64)
    pi, pj = _i64(pi), _i64(pj)
    r = np.empty(len(pi), np.float64)
    _load().or_pearson_pairs(D, D, _p(X), _p(mu), _p(ss), len(pi), _p(pi), _p(pj),
                             1 if kahan else 0, _p(r), n_threads or default_threads())
    return r
