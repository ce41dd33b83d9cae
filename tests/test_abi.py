"""Host-side checks of the C ABI: the library builds, loads and exports every
function include/allpairs.h declares; host helpers agree with the oracle;
argument validation fails cleanly before any device work.  No GPU needed."""
import ctypes
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ap():
    from paper_2009_04755_gb300 import _build
    _build.build()
    import paper_2009_04755_gb300.binding as b
    return b


def test_exports_every_declared_function(ap):
    names = ap.declared_functions()
    assert len(names) >= 12
    L = ctypes.CDLL(ap.LIB_PATH)
    for name in names:
        assert hasattr(L, name), name


def test_status_strings(ap):
    for s in range(7):
        assert ap.status_string(s)
    assert ap.status_string(99) == "unknown status"


@pytest.mark.parametrize("n", [0, 1, 2, 3, 10, 257, 8192])
def test_pair_count_and_index_match_oracle(ap, oracle_lib, n):
    assert ap.pair_count(n) == oracle_lib.pair_count(n)
    if 2 <= n <= 257:
        for i, j in [(0, 1), (0, n - 1), (n - 2, n - 1), (n // 3, n // 2 + 1)]:
            if i < j:
                assert ap.pair_index(i, j, n) == oracle_lib.pair_index(i, j, n)
    assert ap.pair_index(1, 1, max(n, 2)) == -1


def test_pair_index_full_enumeration(ap, oracle_lib):
    n = 37
    pi, pj = oracle_lib.all_pairs(n)
    got = [ap.pair_index(i, j, n) for i, j in zip(pi, pj)]
    assert got == list(range(len(pi)))


@pytest.mark.parametrize("n,block", [(8, 1), (16, 1), (100, 7), (1000, 128), (3, 8)])
def test_plan_tiles_cover_upper_triangle_once(ap, n, block):
    t = ap.plan_tiles(n, block)
    nb = (n + block - 1) // block
    assert len(t) == nb * (nb + 1) // 2
    assert np.all(t[:, 0] <= t[:, 1])
    assert len({(a, b) for a, b in t}) == len(t)


def _morton(i, j, bits):
    k = 0
    for b in range(bits - 1, -1, -1):
        k = (k << 2) | (((i >> b) & 1) << 1) | ((j >> b) & 1)
    return k


@pytest.mark.parametrize("nb", [8, 32])
def test_plan_tiles_quadrant_order(ap, oracle_lib, nb):
    # power-of-two grid: the block order is the Z order of the quadrant split
    t = [tuple(x) for x in ap.plan_tiles(nb, 1)]
    bits = int(np.log2(nb))
    want = sorted([(i, j) for i in range(nb) for j in range(i, nb)],
                  key=lambda p: _morton(p[0], p[1], bits))
    assert t == want
    # and restricted to the strict triangle it is the oracle's order
    oi, oj = oracle_lib.dc_order(nb)
    strict = [p for p in t if p[0] < p[1]]
    assert strict == list(zip(oi.tolist(), oj.tolist()))


def test_plan_tiles_rejects_bad_args(ap):
    cnt = ctypes.c_int64(5)
    L = ap.lib()
    assert L.ap_plan_tiles(-1, 4, None, 0, ctypes.byref(cnt)) == ap.AP_ERR_INVALID_ARG
    assert L.ap_plan_tiles(10, 0, None, 0, ctypes.byref(cnt)) == ap.AP_ERR_INVALID_ARG
    assert L.ap_plan_tiles(10, 4, None, 10, ctypes.byref(cnt)) == ap.AP_ERR_INVALID_ARG
    assert L.ap_plan_tiles(10, 4, None, 0, None) == ap.AP_ERR_INVALID_ARG


def test_invalid_args_rejected_before_device_work(ap):
    L = ap.lib()
    h = ctypes.c_void_p(123)
    assert L.ap_create_items(None, None, ctypes.byref(h)) == ap.AP_ERR_INVALID_ARG
    assert h.value is None
    d = ap.ItemsDesc()
    assert L.ap_create_items(ctypes.byref(d), None, None) == ap.AP_ERR_INVALID_ARG
    d.kind = 7
    assert L.ap_create_items(ctypes.byref(d), None, ctypes.byref(h)) == ap.AP_ERR_INVALID_ARG
    d.kind = ap.AP_ITEMS_VECTOR
    d.n_items = -1
    assert L.ap_create_items(ctypes.byref(d), None, ctypes.byref(h)) == ap.AP_ERR_INVALID_ARG
    # NULL handles
    assert L.ap_run_pairs(None, 0, 0, None, None, None) == ap.AP_ERR_INVALID_ARG
    assert L.ap_backward(None, None, None, None, None, None) == ap.AP_ERR_INVALID_ARG
    assert L.ap_ascent(None, None, 1, 0.1, 0.0, None, None, None) == ap.AP_ERR_INVALID_ARG
    assert L.ap_update_items(None, None, 0, None) == ap.AP_ERR_INVALID_ARG
    assert L.ap_destroy(None) == ap.AP_OK
    assert L.ap_last_device_error(None) == 0
    st = ap.RunStats()
    assert L.ap_get_stats(None, ctypes.byref(st)) == ap.AP_ERR_INVALID_ARG


def test_struct_layouts_match_header(ap, tmp_path):
    """The ctypes mirrors of the ABI structs against the header itself: a C
    program compiled with include/allpairs.h prints sizeof and offsetof of
    every field."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    structs = {"ap_items_desc": ap.ItemsDesc, "ap_run_stats": ap.RunStats, "ap_plan": ap.Plan}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "allpairs.h"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True,
                               check=True).stdout.splitlines():
        cname, field, v = line.split()
        got[(cname, field)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


@pytest.mark.parametrize("n,dim,slots", [(1000, 3000, 3), (4096, 65536, 6), (8192, 3 << 20, 16),
                                         (16384, 3 << 20, 32), (5000, 100, 7), (300, 64, 50)])
def test_out_of_core_schedule_covers_every_macro_pair(ap, n, dim, slots):
    # the library verifies the schedule itself (each macro pair once, both
    # macros resident); here: loads are at least one per macro, exactly one
    # when everything fits, and every loaded byte is a macro of the set
    dp = (dim + 63) // 64 * 64
    cache = slots * 256 * dp * 4
    r = ap.plan_out_of_core(n, dim, cache)
    macros = (n + 255) // 256
    assert r["macros"] == macros
    assert r["slots"] == min(slots, macros)
    assert r["loads"] >= macros
    if slots >= macros:
        assert r["loads"] == macros and r["steps"] == 1
    else:
        assert r["loads"] / macros < 2.5


def test_out_of_core_schedule_rejects_tiny_cache(ap):
    with pytest.raises(ap.APError) as e:
        ap.plan_out_of_core(4096, 1024, 2 * 256 * 1024 * 4)
    assert e.value.status == ap.AP_ERR_INVALID_ARG
