"""GPU parity of the out-of-core Pearson path: vectors stay in page-locked
host memory and stream through the HBM slot cache (the device cache of
Sec. IV-A), checked against the FP64 oracle and the in-HBM path."""
import numpy as np
import pytest

import synth
from gpu_util import PEARSON_ATOL, pearson_tolerance, regroup_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ap():
    import paper_2009_04755_gb300 as ap
    ap.lib()
    return ap


def _slot_bytes(D):
    return 256 * ((D + 63) // 64 * 64) * 4


@pytest.mark.parametrize("n,D,slots", [(1000, 3000, 3), (1100, 2048, 3), (513, 1000, 9)])
def test_out_of_core_all_pairs(ap, oracle_lib, n, D, slots):
    X = synth.vectors_grouped(n, D, seed=n).pin_memory()
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    with ap.Items.from_vectors(X, slot_cache_bytes=slots * _slot_bytes(D)) as it:
        got = it.run_pairs().cpu().numpy()
        st = it.stats()
        again = it.run_pairs().cpu().numpy()
        assert it.last_device_error() == 0
    tol = pearson_tolerance(X.numpy(), pi, pj, 1)
    assert np.all(np.abs(got - ref) <= tol), float(np.abs(got - ref).max())
    np.testing.assert_allclose(again, got, rtol=0, atol=1e-12)
    macros = (n + 255) // 256
    plan = ap.binding.plan_out_of_core(n, D, slots * _slot_bytes(D))
    assert st["reuse_R"] >= 1.0
    assert st["item_loads"] >= n
    if slots >= macros:
        assert st["item_loads"] == n
    assert st["h2d_bytes"] == st["item_loads"] * D * 4
    assert plan["loads"] >= macros


def test_out_of_core_matches_in_hbm_path(ap):
    n, D = 900, 4096
    X = synth.vectors_grouped(n, D, seed=3)
    with ap.Items.from_vectors(X.cuda()) as it:
        r_hbm = it.run_pairs().cpu().numpy()
    with ap.Items.from_vectors(X.pin_memory(), slot_cache_bytes=3 * _slot_bytes(D) + 1) as it:
        r_ooc = it.run_pairs().cpu().numpy()
    # same products; only their grouping into FP32 chains differs (K is split
    # into ranges whose sums meet in FP64)
    pi, pj = np.triu_indices(n, 1)
    assert np.all(np.abs(r_hbm - r_ooc) <= regroup_tolerance(X.numpy(), pi, pj))


def test_out_of_core_coverage(ap):
    n, D = 1300, 64
    X = synth.vectors_grouped(n, D, seed=5).pin_memory()
    with ap.Items.from_vectors(X, slot_cache_bytes=3 * _slot_bytes(D)) as it:
        cnt = it.run_pairs(ap.AP_FN_COVERAGE).cpu().numpy()
    assert cnt.shape == (n * (n - 1) // 2,)
    assert np.all(cnt == 1)


def test_out_of_core_rejects(ap):
    X = torch.randn(600, 128)
    with pytest.raises(ap.APError):           # device data cannot be out of core
        ap.Items.from_vectors(X.cuda(), slot_cache_bytes=1 << 30)
    with pytest.raises(ap.APError):           # fewer than 3 slots for 3 macros
        ap.Items.from_vectors(X.pin_memory(), slot_cache_bytes=_slot_bytes(128))
    with ap.Items.from_vectors(X.pin_memory(), slot_cache_bytes=3 * _slot_bytes(128)) as it:
        with pytest.raises(ap.APError):       # storage is not resident
            it.update(X.cuda())
        with pytest.raises(ap.APError):       # FP32 path is not built out of core
            it.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32)


def test_out_of_core_larger_sampled(ap, oracle_lib):
    n, D = 4096, 65536
    X = synth.vectors_grouped(n, D, seed=11).pin_memory()
    with ap.Items.from_vectors(X, slot_cache_bytes=6 * _slot_bytes(D)) as it:
        r = it.run_pairs()
        torch.cuda.synchronize()
        st = it.stats()
    rng = np.random.default_rng(2)
    pi = rng.integers(0, n - 1, 3000)
    pj = rng.integers(0, n, 3000)
    keep = pi < pj
    pi, pj = pi[keep], pj[keep]
    rows = np.unique(np.concatenate([pi, pj]))
    sub = X.numpy()[rows]
    remap = {v: k for k, v in enumerate(rows)}
    a = np.array([remap[v] for v in pi]); b = np.array([remap[v] for v in pj])
    ref = oracle_lib.pearson(sub, a, b)
    p = torch.from_numpy(pi * n - pi * (pi + 1) // 2 + (pj - pi - 1)).cuda()
    got = r[p].cpu().numpy()
    assert np.all(np.abs(got - ref) <= pearson_tolerance(sub, a, b, 1))
    assert 1.0 < st["reuse_R"] < 2.5


@pytest.mark.parametrize("n,D", [(1000, 3000), (300, 200), (513, 1024)])
def test_load_and_run_matches_separate_calls(ap, oracle_lib, n, D):
    """Transfers overlapped with the Gram macro by macro give the same
    correlations as loading first and running after."""
    X1 = synth.vectors_grouped(n, D, seed=21)
    X2 = synth.vectors_grouped(n, D, seed=22).pin_memory()
    pi, pj = oracle_lib.all_pairs(n)
    with ap.Items.from_vectors(X1.cuda()) as it:
        got = it.load_and_run(X2).cpu().numpy()
        st = it.stats()
        again = it.run_pairs().cpu().numpy()          # the set now holds X2
        assert it.last_device_error() == 0
    ref = oracle_lib.pearson(X2.numpy(), pi, pj)
    assert np.all(np.abs(got - ref) <= pearson_tolerance(X2.numpy(), pi, pj, 1))
    assert np.all(np.abs(got - again) <= regroup_tolerance(X2.numpy(), pi, pj))
    assert st["reuse_R"] == 1.0 and st["h2d_bytes"] == n * D * 4


def test_out_of_core_lru_policy(ap, oracle_lib):
    """The paper's policy (recursive order, LRU eviction) gives the same
    correlations with more loads."""
    n, D = 1300, 1024
    X = synth.vectors_grouped(n, D, seed=31).pin_memory()
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    with ap.Items.from_vectors(X, slot_cache_bytes=3 * _slot_bytes(D)) as it:
        r0 = it.run_pairs().cpu().numpy()
        R0 = it.stats()["reuse_R"]
        it.set_out_of_core_policy(ap.binding.AP_OOC_DC_LRU)
        r1 = it.run_pairs().cpu().numpy()
        R1 = it.stats()["reuse_R"]
        cnt = it.run_pairs(ap.AP_FN_COVERAGE).cpu().numpy()
    tol = pearson_tolerance(X.numpy(), pi, pj, 1)
    assert np.all(np.abs(r0 - ref) <= tol) and np.all(np.abs(r1 - ref) <= tol)
    assert np.all(cnt == 1)
    assert R1 >= R0 >= 1.0


def _slice_cache(n, cols):
    """Cache for column chunks of `cols` columns: two hi/lo chunk buffers and
    the four-piece raw ring."""
    rows = (n + 127) // 128 * 128
    return cols * (2 * 4 * rows + 4 * 256 * min(4, -(-n // 256)))


def test_out_of_core_column_slices(ap, oracle_lib):
    """Column slices (R = 1): rows centred on the mean of their first chunk,
    the Gram accumulated over three chunks (the last one ragged), the exact
    centring recovered at the end; large row-dependent means exercise the
    shifted-data correction."""
    n, D = 1000, 3000
    X = synth.vectors_grouped(n, D, seed=41) + torch.linspace(-3.0, 7.0, n)[:, None]
    X = X.contiguous().pin_memory()
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    tol = pearson_tolerance(X.numpy(), pi, pj, 1)
    cache = max(_slice_cache(n, 1024), 3 * _slot_bytes(D))   # the macro schedule needs 3 slots
    plan = ap.binding.plan_out_of_core(n, D, cache, ap.binding.AP_OOC_K_SLICED)
    assert plan["steps"] == 3 and plan["loads"] == 4
    with ap.Items.from_vectors(X, slot_cache_bytes=cache) as it:
        r0 = it.run_pairs().cpu().numpy()
        it.set_out_of_core_policy(ap.binding.AP_OOC_K_SLICED)
        r2 = it.run_pairs().cpu().numpy()
        st = it.stats()
        again = it.run_pairs().cpu().numpy()
        cnt = it.run_pairs(ap.AP_FN_COVERAGE).cpu().numpy()
        assert it.last_device_error() == 0
        it.set_out_of_core_policy(ap.binding.AP_OOC_RESIDENT_STREAM)
        r0b = it.run_pairs().cpu().numpy()
    assert np.all(np.abs(r2 - ref) <= tol), float(np.abs(r2 - ref).max())
    assert np.all(np.abs(r0 - ref) <= tol)
    assert st["reuse_R"] == 1.0 and st["h2d_bytes"] == n * D * 4
    assert np.abs(again - r2).max() <= 1e-12
    assert np.all(cnt == 1)
    assert np.abs(r0b - r0).max() <= 1e-12
    assert np.all(np.abs(r2 - r0) <= regroup_tolerance(X.numpy(), pi, pj) + 2 * tol)


@pytest.mark.parametrize("n,D", [(300, 200), (257, 4096)])
def test_out_of_core_column_slices_shapes(ap, oracle_lib, n, D):
    X = synth.vectors_grouped(n, D, seed=n + 7).pin_memory()
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    cache = max(_slice_cache(n, 64 * 3), 3 * _slot_bytes(D))
    with ap.Items.from_vectors(X, slot_cache_bytes=cache) as it:
        it.set_out_of_core_policy(ap.binding.AP_OOC_K_SLICED)
        got = it.run_pairs().cpu().numpy()
        assert it.last_device_error() == 0
    assert np.all(np.abs(got - ref) <= pearson_tolerance(X.numpy(), pi, pj, 1))


def test_out_of_core_column_slices_reject_small_cache(ap):
    n, D = 1000, 64
    X = synth.vectors_grouped(n, D, seed=2).pin_memory()
    cache = 3 * _slot_bytes(D)               # three macro slots, not 64 columns of all rows
    assert cache < _slice_cache(n, 64)
    with ap.Items.from_vectors(X, slot_cache_bytes=cache) as it:
        with pytest.raises(ap.APError):
            it.set_out_of_core_policy(ap.binding.AP_OOC_K_SLICED)
        r = it.run_pairs().cpu().numpy()     # the macro schedule is untouched
    assert np.isfinite(r).all()


def test_encoded_items_parse_stage_and_host_cache(ap, oracle_lib):
    """Rows given encoded: parsed on host threads into the pinned host cache
    (the second-level cache), streamed through the device cache.  Without a
    host cache (two staging slots) device-cache reloads mostly decode again;
    with one that holds the set, a second run decodes nothing.  Results equal
    the pinned-array run."""
    n, D = 1000, 3000
    X = synth.vectors_grouped(n, D, seed=61)
    Xn = X.numpy()
    blobs = [ap.binding.encode_vector(Xn[i]) for i in range(n)]
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(Xn, pi, pj)
    tol = pearson_tolerance(Xn, pi, pj, 1)
    cache = 3 * _slot_bytes(D)                       # 3 device slots for 4 macros: R > 1
    with ap.Items.from_vectors(X.pin_memory(), slot_cache_bytes=cache) as it:
        base = it.run_pairs().cpu().numpy()
        loads = it.stats()["item_loads"]
    with ap.Items.from_encoded(blobs, D, slot_cache_bytes=cache, host_cache_bytes=0,
                               parse_threads=4) as it:
        got = it.run_pairs().cpu().numpy()
        st = it.stats()
        assert it.last_device_error() == 0
    assert np.all(np.abs(got - ref) <= tol)
    assert np.abs(got - base).max() <= 1e-12
    # two host slots even without a cache: a reload may still find its macro
    assert st["item_loads"] == loads and n <= st["parsed_rows"] <= loads
    host = 4 * 256 * D * 4                           # every macro decoded fits
    with ap.Items.from_encoded(blobs, D, slot_cache_bytes=cache, host_cache_bytes=host) as it:
        first = it.run_pairs().cpu().numpy()
        s1 = it.stats()
        second = it.run_pairs().cpu().numpy()
        s2 = it.stats()
    assert np.abs(first - base).max() <= 1e-12 and np.abs(second - base).max() <= 1e-12
    assert s1["parsed_rows"] == n and s2["parsed_rows"] == 0
    assert s2["host_hit_rate"] == 1.0 and s1["host_hit_rate"] < 1.0


def test_encoded_items_reject(ap):
    n, D = 300, 256
    X = synth.vectors_grouped(n, D, seed=62).numpy()
    blobs = [ap.binding.encode_vector(X[i]) for i in range(n)]
    cache = 3 * _slot_bytes(D)
    with ap.Items.from_encoded(blobs, D, slot_cache_bytes=cache) as it:
        with pytest.raises(ap.APError):              # slices need raw column ranges
            it.set_out_of_core_policy(ap.binding.AP_OOC_K_SLICED)
    bad = list(blobs)
    bad[7] = bad[7][:-3]                             # a truncated row
    with ap.Items.from_encoded(bad, D, slot_cache_bytes=cache) as it:
        with pytest.raises(ap.APError):
            it.run_pairs()
    with pytest.raises(ap.APError):                  # encoded rows need the out-of-core path
        ap.Items.from_encoded(blobs, D, slot_cache_bytes=0)


def _check_timeline(tr, n_index, copy_bytes):
    """Every task once per index and stage, in issue order on its stream,
    and the dependencies of the pipeline respected on the device clock."""
    eps = 1e-3
    by = {}
    for e in tr:
        assert 0.0 <= e["start_ms"] <= e["end_ms"] + eps
        by.setdefault((e["stage"], e["index"]), []).append(e)
    for stage in ("copy", "preprocess", "gram"):
        assert sorted(i for (s, i) in by if s == stage) == list(range(n_index)), stage
    assert [i for (s, i) in by if s == "finalize"] == [0]
    assert sum(e["bytes"] for e in tr if e["stage"] == "copy") == copy_bytes
    for stream in ("compute", "copy", "preprocess"):
        evs = [e for e in tr if e["stream"] == stream]
        for a, b in zip(evs, evs[1:]):
            assert b["start_ms"] >= a["end_ms"] - eps, stream
    for k in range(n_index):
        c, p, g = by[("copy", k)][0], by[("preprocess", k)][0], by[("gram", k)][0]
        assert p["start_ms"] >= c["start_ms"] - eps
        assert g["start_ms"] >= p["end_ms"] - eps
    fin = by[("finalize", 0)][0]
    assert fin["start_ms"] >= max(e["end_ms"] for e in tr if e["stage"] == "gram") - eps


def test_out_of_core_trace_timeline(ap):
    """The task trace of Sec. IV-C on the column-slice pipeline: per stream,
    per chunk, copies / pre-processing / Gram in order, bytes accounted."""
    n, D = 1000, 3000
    X = synth.vectors_grouped(n, D, seed=5).pin_memory()
    cache = max(_slice_cache(n, 1024), 3 * _slot_bytes(D))
    with ap.Items.from_vectors(X, slot_cache_bytes=cache) as it:
        it.set_out_of_core_policy(ap.binding.AP_OOC_K_SLICED)
        untraced = it.run_pairs().cpu().numpy()
        assert it.trace() == []
        it.set_trace(True)
        got = it.run_pairs().cpu().numpy()
        tr = it.trace()
        it.set_trace(False)
        assert it.trace() == []
    assert np.array_equal(got, untraced)
    _check_timeline(tr, 3, n * D * 4)


def test_load_and_run_trace_timeline(ap):
    n, D = 600, 4096
    X = synth.vectors_grouped(n, D, seed=6)
    with ap.Items.from_vectors(X.cuda()) as it:
        it.set_trace(True)
        it.load_and_run(X.pin_memory())
        tr = it.trace()
    _check_timeline(tr, (n + 255) // 256, n * D * 4)
