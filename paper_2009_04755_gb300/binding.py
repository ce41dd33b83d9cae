"""Thin Python binding of libap.so (the C ABI in include/allpairs.h).

Argument marshalling only: torch supplies device memory and the current CUDA
stream, ctypes passes raw pointers and sizes; every step of the all-pairs
computation runs in the library's CUDA kernels.  There is no CPU fallback:
``lib()`` raises if the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libap.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "allpairs.h")

# ap_status
AP_OK, AP_ERR_INVALID_ARG, AP_ERR_OOM, AP_ERR_CUDA, AP_ERR_TIMEOUT, AP_ERR_UNSUPPORTED, \
    AP_ERR_STATE = range(7)
# ap_item_kind
AP_ITEMS_CLOUD2D, AP_ITEMS_CLOUD3D, AP_ITEMS_VECTOR, AP_ITEMS_SPARSE = range(4)
# ap_pair_fn
AP_FN_OVERLAP, AP_FN_PEARSON, AP_FN_COVERAGE, AP_FN_GMM_L2, AP_FN_BHATTACHARYYA, \
    AP_FN_COSINE = range(6)
# ap_precision
AP_PREC_FP32, AP_PREC_SPLIT_BF16 = range(2)


class ItemsDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("data_on_host", ctypes.c_int32),
                ("n_items", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("weight", ctypes.c_void_p),
                ("data", ctypes.c_void_p), ("dim", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("precisions", ctypes.c_uint32), ("slot_cache_bytes", ctypes.c_uint64),
                ("indices", ctypes.c_void_p), ("blobs", ctypes.c_void_p),
                ("blob_bytes", ctypes.c_void_p), ("codec", ctypes.c_int32),
                ("parse_threads", ctypes.c_int32), ("host_cache_bytes", ctypes.c_uint64)]


class RunStats(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_int64), ("item_loads", ctypes.c_int64),
                ("reuse_R", ctypes.c_double), ("h2d_bytes", ctypes.c_uint64),
                ("slot_hit_rate", ctypes.c_double), ("tile_m", ctypes.c_int32),
                ("tile_n", ctypes.c_int32), ("order", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("parsed_rows", ctypes.c_int64),
                ("host_hit_rate", ctypes.c_double)]


class Plan(ctypes.Structure):
    _fields_ = [("block_items", ctypes.c_int32), ("block_pts", ctypes.c_int32),
                ("reg_r", ctypes.c_int32), ("sorted", ctypes.c_int32), ("rate", ctypes.c_double),
                ("k_split", ctypes.c_int32), ("mma_ctas", ctypes.c_int32)]


class TraceEvent(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_int32), ("stage", ctypes.c_int32), ("index", ctypes.c_int64),
                ("bytes", ctypes.c_uint64), ("start_ms", ctypes.c_double),
                ("end_ms", ctypes.c_double)]


STAGE_NAMES = ("copy", "preprocess", "gram", "finalize")
STREAM_NAMES = ("compute", "copy", "preprocess")


class APError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


_lib = None


def lib():
    """Load libap.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libap.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        sig = {
            "ap_encode_vector": (i32, [vp, i64, i32, vp, ctypes.c_uint64, vp]),
            "ap_decode_vector": (i32, [vp, ctypes.c_uint64, i32, i64, vp]),
            "ap_create_items": (i32, [ctypes.POINTER(ItemsDesc), vp, ctypes.POINTER(vp)]),
            "ap_update_items": (i32, [vp, vp, i32, vp]),
            "ap_run_pairs": (i32, [vp, i32, i32, vp, vp, vp]),
            "ap_backward": (i32, [vp, vp, vp, vp, vp, vp]),
            "ap_ascent": (i32, [vp, vp, i32, f32, f32, vp, vp, vp]),
            "ap_destroy": (i32, [vp]),
            "ap_get_stats": (i32, [vp, ctypes.POINTER(RunStats)]),
            "ap_status_string": (ctypes.c_char_p, [i32]),
            "ap_last_cuda_error": (ctypes.c_char_p, []),
            "ap_last_device_error": (i32, [vp]),
            "ap_pair_count": (i64, [i64]),
            "ap_pair_index": (i64, [i64, i64, i64]),
            "ap_plan_tiles": (i32, [i64, i32, vp, i64, ctypes.POINTER(i64)]),
            "ap_tune": (i32, [vp, i32, vp, ctypes.POINTER(Plan)]),
            "ap_get_plan": (i32, [vp, ctypes.POINTER(Plan)]),
            "ap_set_debug": (i32, [vp, i32, ctypes.c_uint64]),
            "ap_load_and_run": (i32, [vp, vp, vp, vp]),
            "ap_set_plan": (i32, [vp, ctypes.POINTER(Plan)]),
            "ap_plan_out_of_core": (i32, [i64, i64, ctypes.c_uint64, i32, ctypes.POINTER(i64),
                                          ctypes.POINTER(i64), ctypes.POINTER(i64)]),
            "ap_set_out_of_core_policy": (i32, [vp, i32]),
            "ap_run_pairs_list": (i32, [vp, i32, i32, vp, vp, i64, vp, vp, vp]),
            "ap_backward_list": (i32, [vp, vp, vp, i64, vp, vp, vp, vp, vp]),
            "ap_ascent_list": (i32, [vp, vp, vp, i64, vp, i32, f32, f32, vp, vp, vp]),
            "ap_set_trace": (i32, [vp, i32]),
            "ap_get_trace": (i32, [vp, ctypes.POINTER(TraceEvent), i64, ctypes.POINTER(i64)]),
            "ap_pipe_rate": (i32, [i32, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_functions() -> list[str]:
    """Names of the functions include/allpairs.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ap_[a-z_]+)\s*\(", text)))


def status_string(s: int) -> str:
    return lib().ap_status_string(int(s)).decode()


def check(status: int, what: str):
    if status != AP_OK:
        if status in (AP_ERR_OOM, AP_ERR_CUDA):
            cuda = lib().ap_last_cuda_error().decode()
            if cuda:
                what = f"{what} [{cuda}]"
        raise APError(status, what)


def pair_count(n: int) -> int:
    return int(lib().ap_pair_count(int(n)))


def pair_index(i: int, j: int, n: int) -> int:
    return int(lib().ap_pair_index(int(i), int(j), int(n)))


PIPE_FMA, PIPE_EX2, PIPE_RCP, PIPE_FMA2 = 0, 1, 2, 3


def pipe_rate(pipe: int) -> dict:
    """Measured issue rate of one SM pipe on the current device
    (ap_pipe_rate): results per clock per SM, per second, and the SM clock
    seen during the probe."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(lib().ap_pipe_rate(int(pipe), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
          "ap_pipe_rate")
    return {"per_clk_per_sm": a.value, "per_s": b.value, "sm_mhz": c.value}


def plan_tiles(n: int, block: int):
    """Upper-triangle block pairs (I, J) in recursive quadrant order (host)."""
    import numpy as np
    cnt = ctypes.c_int64(0)
    check(lib().ap_plan_tiles(int(n), int(block), None, 0, ctypes.byref(cnt)), "ap_plan_tiles")
    out = np.empty(2 * max(cnt.value, 1), np.int32)
    check(lib().ap_plan_tiles(int(n), int(block), out.ctypes.data, cnt.value, ctypes.byref(cnt)),
          "ap_plan_tiles")
    return out[:2 * cnt.value].reshape(-1, 2)


AP_OOC_RESIDENT_STREAM, AP_OOC_DC_LRU, AP_OOC_K_SLICED = 0, 1, 2
AP_CODEC_NONE, AP_CODEC_XOR_VARINT = 0, 1


def encode_vector(x, codec: int = AP_CODEC_XOR_VARINT) -> bytes:
    """Encode one row (float32) for the parse stage."""
    import numpy as np
    x = np.ascontiguousarray(x, np.float32)
    cap = ctypes.c_uint64()
    check(lib().ap_encode_vector(x.ctypes.data, x.size, codec, None, 0, ctypes.byref(cap)),
          "ap_encode_vector")
    buf = (ctypes.c_uint8 * max(cap.value, 1))()
    n = ctypes.c_uint64()
    check(lib().ap_encode_vector(x.ctypes.data, x.size, codec, buf, cap.value, ctypes.byref(n)),
          "ap_encode_vector")
    return ctypes.string_at(buf, n.value)


def decode_vector(blob: bytes, dim: int, codec: int = AP_CODEC_XOR_VARINT):
    import numpy as np
    x = np.empty(dim, np.float32)
    src = (ctypes.c_uint8 * max(len(blob), 1)).from_buffer_copy(blob or b"\0")
    check(lib().ap_decode_vector(src, len(blob), codec, dim, x.ctypes.data), "ap_decode_vector")
    return x


def plan_out_of_core(n: int, dim: int, slot_cache_bytes: int, policy: int = 0) -> dict:
    """Host-only preview of the out-of-core schedule (slots, loads, steps)."""
    s, l, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(lib().ap_plan_out_of_core(int(n), int(dim), int(slot_cache_bytes), int(policy),
                                    ctypes.byref(s), ctypes.byref(l), ctypes.byref(t)),
          "ap_plan_out_of_core")
    return {"slots": s.value, "loads": l.value, "steps": t.value,
            "macros": (int(n) + 255) // 256}


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Items:
    """A library-owned item set (``ap_items*``)."""

    def __init__(self, handle, kind: int, n: int):
        self._h = handle
        self.kind = kind
        self.n = n
        self.P = n * (n - 1) // 2 if n >= 2 else 0
        self._keep = []

    # ---- construction -------------------------------------------------
    @classmethod
    def from_clouds(cls, clouds: dict, device: str = "cuda", stream=None,
                    sync: bool = True) -> "Items":
        """Clouds dict (numpy or torch): dim, offsets, x, y, z, sigma, weight.
        device "cuda": the arrays are copied to the device first; "cpu": the
        library copies them from (pinned) host memory itself.  The creation
        runs on `stream` (default: torch's current stream); sync=False
        returns without waiting for it (the host arrays are kept alive by the
        handle until it is closed)."""
        import numpy as np
        import torch
        dim = int(clouds["dim"])
        off = np.ascontiguousarray(np.asarray(clouds["offsets"]), dtype=np.int64)
        n = len(off) - 1

        def dev(a):
            if a is None:
                return None
            t = torch.as_tensor(np.asarray(a) if not torch.is_tensor(a) else a)
            t = t.to(device=device, dtype=torch.float32).contiguous()
            return t.pin_memory() if device == "cpu" else t

        arrs = {k: dev(clouds.get(k)) for k in ("x", "y", "z", "sigma", "weight")}
        if dim != 3:
            arrs["z"] = None
        d = ItemsDesc()
        d.kind = AP_ITEMS_CLOUD3D if dim == 3 else AP_ITEMS_CLOUD2D
        d.data_on_host = 1 if device == "cpu" else 0
        d.n_items = n
        d.offsets = off.ctypes.data
        for k, t in arrs.items():
            setattr(d, k, None if t is None else t.data_ptr())
        if device != "cpu":
            # the copies above ran on torch's current stream
            ev = torch.cuda.Event()
            ev.record()
            (stream or torch.cuda.current_stream()).wait_event(ev)
        h = ctypes.c_void_p()
        check(lib().ap_create_items(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)),
              "ap_create_items")
        if sync:
            torch.cuda.synchronize()
        obj = cls(h, d.kind, n)
        obj._keep = (arrs, off)                 # sources until the handle is closed
        return obj

    @classmethod
    def from_vectors(cls, X, precisions=(AP_PREC_SPLIT_BF16,), stream=None,
                     slot_cache_bytes: int = 0) -> "Items":
        """X: torch float32 [n, D] on the GPU, or on the host (ideally pinned).
        slot_cache_bytes > 0 (host X only): out-of-core mode; X must stay alive
        (and unchanged between runs unless that is intended) while the handle
        exists."""
        import torch
        assert X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
        d = ItemsDesc()
        d.kind = AP_ITEMS_VECTOR
        d.data_on_host = 0 if X.is_cuda else 1
        d.n_items = X.shape[0]
        d.data = X.data_ptr()
        d.dim = X.shape[1]
        d.ld = X.stride(0)
        d.precisions = sum(1 << p for p in precisions)
        d.slot_cache_bytes = int(slot_cache_bytes)
        h = ctypes.c_void_p()
        check(lib().ap_create_items(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)),
              "ap_create_items")
        obj = cls(h, AP_ITEMS_VECTOR, X.shape[0])
        if slot_cache_bytes:
            obj._keep.append(X)          # the library reads it on every run
        return obj

    @classmethod
    def from_sparse(cls, offsets, indices, values, dim: int, stream=None) -> "Items":
        """Sparse rows in CSR form: offsets int64 [n+1] (host), indices int32
        (strictly increasing per row, < dim) and values float32 as numpy arrays
        (copied from the host) or torch tensors (host or GPU)."""
        import numpy as np
        import torch
        off = np.ascontiguousarray(np.asarray(offsets), dtype=np.int64)
        n = len(off) - 1

        def arr(a, dt):
            t = a if torch.is_tensor(a) else torch.from_numpy(np.ascontiguousarray(a))
            return t.to(dtype=dt).contiguous()

        idx, val = arr(indices, torch.int32), arr(values, torch.float32)
        d = ItemsDesc()
        d.kind = AP_ITEMS_SPARSE
        d.data_on_host = 0 if idx.is_cuda else 1
        assert idx.is_cuda == val.is_cuda
        d.n_items = n
        d.offsets = off.ctypes.data
        d.indices = idx.data_ptr() if idx.numel() else None
        d.data = val.data_ptr() if val.numel() else None
        d.dim = int(dim)
        h = ctypes.c_void_p()
        check(lib().ap_create_items(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)),
              "ap_create_items")
        return cls(h, AP_ITEMS_SPARSE, n)

    @classmethod
    def from_encoded(cls, blobs, dim: int, slot_cache_bytes: int, host_cache_bytes: int = 0,
                     parse_threads: int = 0, codec: int = AP_CODEC_XOR_VARINT,
                     stream=None) -> "Items":
        """Out-of-core vector set whose rows arrive encoded (a list of bytes,
        one per row); the library parses them on host threads into a pinned
        host cache of host_cache_bytes and streams them through an HBM slot
        cache of slot_cache_bytes."""
        n = len(blobs)
        bufs = [(ctypes.c_uint8 * max(len(b), 1)).from_buffer_copy(b or b"\0") for b in blobs]
        ptrs = (ctypes.c_void_p * max(n, 1))(*[ctypes.addressof(b) for b in bufs])
        lens = (ctypes.c_uint64 * max(n, 1))(*[len(b) for b in blobs])
        d = ItemsDesc()
        d.kind = AP_ITEMS_VECTOR
        d.data_on_host = 1
        d.n_items = n
        d.dim = int(dim)
        d.precisions = 1 << AP_PREC_SPLIT_BF16
        d.slot_cache_bytes = int(slot_cache_bytes)
        d.blobs = ctypes.addressof(ptrs)
        d.blob_bytes = ctypes.addressof(lens)
        d.codec = int(codec)
        d.parse_threads = int(parse_threads)
        d.host_cache_bytes = int(host_cache_bytes)
        h = ctypes.c_void_p()
        check(lib().ap_create_items(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)),
              "ap_create_items")
        obj = cls(h, AP_ITEMS_VECTOR, n)
        obj._keep += [bufs, ptrs, lens]      # the library reads them on every run
        return obj

    def update(self, X, stream=None):
        check(lib().ap_update_items(self._h, _ptr(X), 0 if X.is_cuda else 1, _stream_ptr(stream)),
              "ap_update_items")

    # ---- compute ------------------------------------------------------
    def run_pairs(self, fn: int = None, precision: int = AP_PREC_SPLIT_BF16, params=None,
                  out=None, stream=None):
        import torch
        if fn is None:
            fn = {AP_ITEMS_VECTOR: AP_FN_PEARSON, AP_ITEMS_SPARSE: AP_FN_COSINE}.get(
                self.kind, AP_FN_OVERLAP)
        if out is None:
            dt = {AP_FN_OVERLAP: torch.float32, AP_FN_GMM_L2: torch.float32,
                  AP_FN_BHATTACHARYYA: torch.float32, AP_FN_PEARSON: torch.float64,
                  AP_FN_COSINE: torch.float64,
                  AP_FN_COVERAGE: torch.int32}[fn]
            out = (torch.zeros if fn == AP_FN_COVERAGE else torch.empty)(
                max(self.P, 1), dtype=dt, device="cuda")
        check(lib().ap_run_pairs(self._h, fn, precision, _ptr(params), _ptr(out),
                                 _stream_ptr(stream)), "ap_run_pairs")
        return out[:self.P]

    @staticmethod
    def _pair_list(pi, pj):
        import numpy as np
        a = np.ascontiguousarray(np.asarray(pi, dtype=np.int32))
        b = np.ascontiguousarray(np.asarray(pj, dtype=np.int32))
        assert a.shape == b.shape and a.ndim == 1
        return a, b

    def run_pairs_list(self, pi, pj, fn: int = None, precision: int = AP_PREC_SPLIT_BF16,
                       params=None, out=None, stream=None):
        """f for the listed pairs (original item ids, host arrays):
        out[k] = f(pi[k], pj[k]); a transform acts on pj[k]."""
        import torch
        a, b = self._pair_list(pi, pj)
        if fn is None:
            fn = {AP_ITEMS_VECTOR: AP_FN_PEARSON, AP_ITEMS_SPARSE: AP_FN_COSINE}.get(
                self.kind, AP_FN_OVERLAP)
        if out is None:
            dt = torch.float64 if fn in (AP_FN_PEARSON, AP_FN_COSINE) else torch.float32
            out = torch.empty(max(len(a), 1), dtype=dt, device="cuda")
        check(lib().ap_run_pairs_list(self._h, fn, precision, a.ctypes.data, b.ctypes.data,
                                      len(a), _ptr(params), _ptr(out), _stream_ptr(stream)),
              "ap_run_pairs_list")
        return out[:len(a)]

    def backward_list(self, pi, pj, params=None, grad_out=None, stream=None):
        import torch
        a, b = self._pair_list(pi, pj)
        g = torch.empty(max(len(a), 1), 3, dtype=torch.float32, device="cuda")
        f = torch.empty(max(len(a), 1), dtype=torch.float32, device="cuda")
        check(lib().ap_backward_list(self._h, a.ctypes.data, b.ctypes.data, len(a), _ptr(params),
                                     _ptr(grad_out), _ptr(g), _ptr(f), _stream_ptr(stream)),
              "ap_backward_list")
        return g[:len(a)], f[:len(a)]

    def ascent_list(self, pi, pj, params, n_steps: int, eta: float, fmin: float = 1e-30,
                    stream=None):
        import torch
        a, b = self._pair_list(pi, pj)
        f = torch.empty(max(len(a), 1), dtype=torch.float32, device="cuda")
        flags = torch.zeros(max(len(a), 1), dtype=torch.int32, device="cuda")
        check(lib().ap_ascent_list(self._h, a.ctypes.data, b.ctypes.data, len(a), _ptr(params),
                                   int(n_steps), float(eta), float(fmin), _ptr(f), _ptr(flags),
                                   _stream_ptr(stream)), "ap_ascent_list")
        return params, f[:len(a)], flags[:len(a)]

    def load_and_run(self, X_host, out=None, stream=None):
        """Load new host vectors and correlate all pairs, transfers overlapped
        with the Gram (split-BF16)."""
        import torch
        assert not X_host.is_cuda and X_host.dtype == torch.float32
        if out is None:
            out = torch.empty(max(self.P, 1), dtype=torch.float64, device="cuda")
        check(lib().ap_load_and_run(self._h, _ptr(X_host), _ptr(out), _stream_ptr(stream)),
              "ap_load_and_run")
        return out[:self.P]

    def backward(self, params=None, grad_out=None, f_out=None, stream=None):
        import torch
        g = torch.empty(max(self.P, 1), 3, dtype=torch.float32, device="cuda")
        if f_out is None:
            f_out = torch.empty(max(self.P, 1), dtype=torch.float32, device="cuda")
        check(lib().ap_backward(self._h, _ptr(params), _ptr(grad_out), _ptr(g), _ptr(f_out),
                                _stream_ptr(stream)), "ap_backward")
        return g[:self.P], f_out[:self.P]

    def ascent(self, params, n_steps: int, eta: float, fmin: float = 1e-30, stream=None):
        import torch
        f = torch.empty(max(self.P, 1), dtype=torch.float32, device="cuda")
        flags = torch.zeros(max(self.P, 1), dtype=torch.int32, device="cuda")
        check(lib().ap_ascent(self._h, _ptr(params), int(n_steps), float(eta), float(fmin),
                              _ptr(f), _ptr(flags), _stream_ptr(stream)), "ap_ascent")
        return params, f[:self.P], flags[:self.P]

    def tune(self, mode: int = 0, stream=None) -> dict:
        """Autotune the tile plan (clouds); returns the chosen plan."""
        p = Plan()
        check(lib().ap_tune(self._h, int(mode), _stream_ptr(stream), ctypes.byref(p)), "ap_tune")
        return {k: getattr(p, k) for k, _ in Plan._fields_}

    def plan(self) -> dict:
        p = Plan()
        check(lib().ap_get_plan(self._h, ctypes.byref(p)), "ap_get_plan")
        return {k: getattr(p, k) for k, _ in Plan._fields_}

    def set_plan(self, block_items: int, block_pts: int, reg_r: int = 0, k_split: int = 0,
                 mma_ctas: int = 0):
        """Clouds: tile plan (block_items, block_pts, reg_r).  Vector sets:
        (128, 256), k_split (the split-BF16 Gram's column ranges) and
        mma_ctas (1: one CTA per tile, 2 or 0: CTA pairs)."""
        p = Plan(int(block_items), int(block_pts), int(reg_r), 0, 0.0, int(k_split),
                 int(mma_ctas))
        check(lib().ap_set_plan(self._h, ctypes.byref(p)), "ap_set_plan")

    def stats(self) -> dict:
        st = RunStats()
        check(lib().ap_get_stats(self._h, ctypes.byref(st)), "ap_get_stats")
        return {k: getattr(st, k) for k, _ in RunStats._fields_}

    def set_out_of_core_policy(self, policy: int):
        """0: resident set + streamed groups (default); 1: the paper's
        recursive order with LRU eviction; 2: column slices (R = 1)."""
        check(lib().ap_set_out_of_core_policy(self._h, int(policy)), "ap_set_out_of_core_policy")

    def set_trace(self, on: bool = True):
        """Record the tasks of later streamed runs (out-of-core, load-and-run)
        per stream with CUDA events (ap_set_trace)."""
        check(lib().ap_set_trace(self._h, 1 if on else 0), "ap_set_trace")

    def trace(self) -> list:
        """The last traced call's tasks as dicts: stream, stage, index, bytes,
        start_ms, end_ms (ap_get_trace; waits for them)."""
        n = ctypes.c_int64()
        check(lib().ap_get_trace(self._h, None, 0, ctypes.byref(n)), "ap_get_trace")
        buf = (TraceEvent * max(n.value, 1))()
        check(lib().ap_get_trace(self._h, buf, n.value, ctypes.byref(n)), "ap_get_trace")
        return [{"stream": STREAM_NAMES[e.stream], "stage": STAGE_NAMES[e.stage],
                 "index": e.index, "bytes": e.bytes, "start_ms": e.start_ms,
                 "end_ms": e.end_ms} for e in buf[:n.value]]

    def set_debug(self, flags: int, wait_budget_ns: int = 0):
        """Failure-path switch (testing) and device wait budget (0 = 2 s)."""
        check(lib().ap_set_debug(self._h, int(flags), int(wait_budget_ns)), "ap_set_debug")

    def last_device_error(self) -> int:
        return int(lib().ap_last_device_error(self._h))

    def close(self):
        if self._h is not None and self._h.value:
            check(lib().ap_destroy(self._h), "ap_destroy")
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
