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
