"""Host-side checks of the two out-of-core schedules (no GPU): both compute
every macro pair exactly once with both macros resident (the library checks
that itself), the loads per item R (Sec. VI-A) never exceed the LRU policy's
for the schedule-aware policy, and both reach R = 1 when the set fits."""
import pytest


@pytest.fixture(scope="module")
def ap():
    from paper_2009_04755_gb300 import _build
    _build.build()
    import paper_2009_04755_gb300.binding as b
    return b


@pytest.mark.parametrize("n", [1000, 8192, 5000])
def test_policies_cover_and_compare(ap, n):
    D = 4096
    slot = 256 * D * 4
    macros = (n + 255) // 256
    prev = None
    for S in range(3, macros + 2):
        r0 = ap.plan_out_of_core(n, D, S * slot, ap.AP_OOC_RESIDENT_STREAM)
        r1 = ap.plan_out_of_core(n, D, S * slot, ap.AP_OOC_DC_LRU)
        assert r0["loads"] >= macros and r1["loads"] >= macros
        assert r0["loads"] <= r1["loads"]
        if S >= macros:
            assert r0["loads"] == macros and r1["loads"] == macros
        if prev is not None:
            assert r0["loads"] <= prev          # a bigger cache never loads more
        prev = r0["loads"]


def test_policy_rejects_unknown(ap):
    with pytest.raises(ap.APError):
        ap.plan_out_of_core(1000, 64, 10 * 256 * 64 * 4, 7)


def _slices(n, Dp, budget):
    """The column-slice geometry: two hi/lo chunk buffers of all rows and a
    ring of 256-row raw pieces (a whole chunk when that still leaves chunks
    of >= 64K columns, else four pieces)."""
    rows = -(-n // 128) * 128
    pieces = -(-n // 256)
    for r in (pieces, min(pieces, 4)):
        cmax = budget // (2 * 4 * rows + 4 * 256 * r) // 64 * 64
        if cmax >= min(Dp, 65536) or (r == min(pieces, 4) and cmax >= 64):
            count = max(-(-Dp // cmax), min(12, Dp // 262144))  # >= 12 chunks of >= 256K columns
            return count, -(-(-(-Dp // count)) // 64) * 64
    return None


def test_column_slices_plan(ap):
    """Column slices: two chunk buffers, every macro loaded once (R = 1), one
    step per column chunk; chunks shrink as the cache does."""
    n, D = 8192, 3 << 20
    macros = (n + 255) // 256
    p = ap.plan_out_of_core(n, D, 48 << 30, ap.AP_OOC_K_SLICED)
    assert p["slots"] == 2 and p["loads"] == macros
    assert p["steps"] == _slices(n, D, 48 << 30)[0] == 12
    small = ap.plan_out_of_core(n, D, 12 << 30, ap.AP_OOC_K_SLICED)
    assert small["steps"] == _slices(n, D, 12 << 30)[0] > p["steps"]
    assert small["loads"] == macros
    lru = ap.plan_out_of_core(n, D, 48 << 30, ap.AP_OOC_RESIDENT_STREAM)
    assert lru["loads"] > p["loads"]
    with pytest.raises(ap.APError):
        ap.plan_out_of_core(n, D, 1 << 20, ap.AP_OOC_K_SLICED)
