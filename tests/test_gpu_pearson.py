"""GPU parity of the Pearson path (split-BF16 tcgen05 Gram and plain FP32
Gram, FP64 normalisation) against the FP64 oracle, through the C ABI."""
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


def _run(ap, X, prec, precisions=None, host=False):
    precisions = precisions or (prec,)
    src = X.pin_memory() if host else X.cuda()
    with ap.Items.from_vectors(src, precisions=precisions) as it:
        out = it.run_pairs(ap.AP_FN_PEARSON, prec).cpu().numpy()
        assert it.last_device_error() == 0
    return out


@pytest.mark.parametrize("n,D", [(300, 1000), (257, 64), (129, 2050), (2, 2), (40, 20000)])
def test_pearson_all_pairs_match_oracle(ap, oracle_lib, n, D):
    X = synth.vectors_grouped(n, D, seed=n + D)
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    both = (ap.AP_PREC_SPLIT_BF16, ap.AP_PREC_FP32)
    for prec in both:
        got = _run(ap, X, prec, precisions=both)
        tol = pearson_tolerance(X.numpy(), pi, pj, prec)
        over = np.abs(got - ref) > tol
        assert not over.any(), f"prec {prec}: {over.sum()} pairs beyond tolerance, " \
            f"max |err| {np.abs(got - ref).max():.3e}"
        if D >= 16384:
            assert np.abs(got - ref).max() <= PEARSON_ATOL


@pytest.mark.parametrize("D", [4096, 1 << 16])
def test_pearson_strongly_correlated(ap, oracle_lib, D):
    # long correlated chains: the accumulation must not drift (a single FP32
    # tensor-core chain over D would be biased by ~2^-23 D/64 relative)
    n = 64
    g = torch.Generator().manual_seed(3)
    base = torch.randn(1, D, generator=g)
    X = (base + 0.1 * torch.randn(n, D, generator=g)).float()
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    got = _run(ap, X, ap.AP_PREC_SPLIT_BF16)
    assert ref.min() > 0.98
    assert np.all(np.abs(got - ref) <= pearson_tolerance(X.numpy(), pi, pj, 1))
    if D >= 16384:
        assert np.abs(got - ref).max() <= PEARSON_ATOL


def test_pearson_host_source_equals_device_source(ap):
    n, D = 200, 3000
    X = synth.vectors_grouped(n, D, seed=9)
    a = _run(ap, X, ap.AP_PREC_SPLIT_BF16, host=False)
    b = _run(ap, X, ap.AP_PREC_SPLIT_BF16, host=True)
    assert np.array_equal(a, b)


def test_pearson_update_items_reuses_storage(ap, oracle_lib):
    n, D = 150, 512
    X1 = synth.vectors_grouped(n, D, seed=1)
    X2 = synth.vectors_grouped(n, D, seed=2)
    pi, pj = oracle_lib.all_pairs(n)
    with ap.Items.from_vectors(X1.cuda()) as it:
        it.update(X2.cuda())
        got = it.run_pairs().cpu().numpy()
    ref = oracle_lib.pearson(X2.numpy(), pi, pj)
    assert np.all(np.abs(got - ref) <= pearson_tolerance(X2.numpy(), pi, pj, 1))


@pytest.mark.parametrize("prec", [1, 0])
def test_pearson_coverage_every_pair_once(ap, prec, oracle_lib):
    n, D = 777, 64
    X = synth.vectors_grouped(n, D, seed=4)
    with ap.Items.from_vectors(X.cuda(), precisions=(prec,)) as it:
        cnt = it.run_pairs(ap.AP_FN_COVERAGE, prec).cpu().numpy()
    assert cnt.shape == (oracle_lib.pair_count(n),)
    assert np.all(cnt == 1)


def test_pearson_edge_cases(ap):
    # n < 2: nothing to do
    for n in (0, 1):
        X = torch.randn(max(n, 1), 16)[:n].contiguous()
        with ap.Items.from_vectors(X.cuda()) as it:
            assert it.run_pairs().numel() == 0
    # zero-variance item gives NaN for its pairs only
    X = torch.randn(5, 100)
    X[2] = 3.0
    with ap.Items.from_vectors(X.cuda()) as it:
        r = it.run_pairs().cpu().numpy()
    bad = [ap.pair_index(i, 2, 5) for i in range(2)] + [ap.pair_index(2, j, 5) for j in (3, 4)]
    assert np.all(np.isnan(r[bad]))
    good = np.setdiff1d(np.arange(10), bad)
    assert np.all(np.isfinite(r[good]))


def test_pearson_rejects_bad_requests(ap):
    X = torch.randn(10, 64)
    with ap.Items.from_vectors(X.cuda(), precisions=(ap.AP_PREC_SPLIT_BF16,)) as it:
        with pytest.raises(ap.APError) as e:
            it.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32)   # representation not built
        assert e.value.status == 6
        with pytest.raises(ap.APError) as e:
            it.run_pairs(ap.AP_FN_OVERLAP)
        assert e.value.status == 1


def _sample_pairs(n, rng, n_random=1500):
    i, j = [], []
    # all pairs of two random 128 x 256 tiles and one diagonal tile
    for _ in range(2):
        a0 = int(rng.integers(0, n // 128)) * 128
        b0 = int(rng.integers(a0 // 256, n // 256)) * 256
        for a in range(a0, a0 + 128, 9):
            for b in range(b0, b0 + 256, 17):
                if a < b:
                    i.append(a); j.append(b)
    d0 = int(rng.integers(0, n // 256)) * 256
    for a in range(d0, d0 + 256, 11):
        for b in range(a + 1, d0 + 256, 13):
            i.append(a); j.append(b)
    # first row, the last two rows
    for b in range(1, n, 97):
        i.append(0); j.append(b)
    i.append(n - 2); j.append(n - 1)
    a = rng.integers(0, n - 1, n_random)
    b = rng.integers(0, n, n_random)
    keep = a < b
    i.extend(a[keep].tolist()); j.extend(b[keep].tolist())
    return np.array(i, np.int64), np.array(j, np.int64)


def test_pearson_full_size_sampled(ap, oracle_lib):
    """The benchmark's workload (8192 vectors of 2^20 FP32, groups of 16) in
    the benchmark's launch configuration, checked on sampled pairs."""
    n, D = 8192, 1 << 20
    X = synth.vectors_grouped(n, D, seed=0, device="cuda")
    both = (ap.AP_PREC_SPLIT_BF16, ap.AP_PREC_FP32)
    with ap.Items.from_vectors(X, precisions=both) as it:
        r_tc = it.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_SPLIT_BF16)
        r_32 = it.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32)
        torch.cuda.synchronize()
        assert it.last_device_error() == 0
        rng = np.random.default_rng(0)
        pi, pj = _sample_pairs(n, rng)
        rows = np.unique(np.concatenate([pi, pj]))
        sub = X[torch.from_numpy(rows).cuda()].cpu().numpy()
        remap = {r: k for k, r in enumerate(rows)}
        ref = oracle_lib.pearson(sub, [remap[a] for a in pi], [remap[b] for b in pj])
        p = torch.from_numpy(pi * n - pi * (pi + 1) // 2 + (pj - pi - 1)).cuda()
        got_tc = r_tc[p].cpu().numpy()
        got_32 = r_32[p].cpu().numpy()
        assert np.abs(got_tc - ref).max() <= PEARSON_ATOL
        assert np.abs(got_32 - ref).max() <= PEARSON_ATOL
        assert torch.isfinite(r_tc).all() and torch.isfinite(r_32).all()
        # every correlation is a correlation
        assert float(r_tc.abs().max()) <= 1.0


@pytest.mark.parametrize("n,D,ks", [(1000, 3000, [1, 3, 16]), (130, 200, [64]),
                                    (300, 20000, [1, 2])])
def test_pearson_k_split_schedule(ap, oracle_lib, n, D, ks):
    """Split-K units in waves give the whole-tile result: the same products,
    only the grouping of the FP32 chain sums into FP64 differs."""
    X = synth.vectors_grouped(n, D, seed=5 * n + D)
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    tol = pearson_tolerance(X.numpy(), pi, pj, 1)
    tol_regroup = regroup_tolerance(X.numpy(), pi, pj)
    with ap.Items.from_vectors(X.cuda()) as it:
        default = it.plan()["k_split"]
        assert default >= 0
        it.set_plan(128, 256, 0, 0)
        base = it.run_pairs().cpu().numpy()
        assert np.all(np.abs(base - ref) <= tol)
        for k in ks + [-1]:
            it.set_plan(128, 256, 0, k)
            assert it.plan()["k_split"] == (default if k < 0 else k)
            got = it.run_pairs().cpu().numpy()
            assert it.last_device_error() == 0
            assert np.all(np.abs(got - ref) <= tol), float(np.abs(got - ref).max())
            assert np.all(np.abs(got - base) <= tol_regroup)
            cnt = it.run_pairs(ap.AP_FN_COVERAGE).cpu().numpy()
            assert np.all(cnt == 1)
        it.set_plan(128, 256, 0, 0)
        again = it.run_pairs().cpu().numpy()
        np.testing.assert_array_equal(again, base)
        for bad in [(128, 256, 0, -2), (128, 256, 0, 10 ** 6), (64, 256, 0, 4)]:
            with pytest.raises(ap.APError):
                it.set_plan(*bad)


@pytest.mark.parametrize("k_split", [0, -1])
def test_pearson_correlated_bias(ap, oracle_lib, k_split):
    """Strongly correlated and anti-correlated pairs over long vectors: the
    tensor core's truncating accumulation biases each chain toward zero in
    proportion to its length (~9e-7 for unseeded 256-column chains at
    r ~ 0.99); seeded chains must keep the mean error of either sign within
    3e-7 and every pair within 1e-6."""
    n, D = 32, 1 << 18
    g = torch.Generator().manual_seed(11)
    base = torch.randn(1, D, generator=g)
    sign = torch.where(torch.rand(n, 1, generator=g) < 0.5, -1.0, 1.0)
    X = (sign * base + 0.05 * torch.randn(n, D, generator=g)).float()
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    with ap.Items.from_vectors(X.cuda()) as it:
        it.set_plan(128, 256, 0, k_split)
        got = it.run_pairs().cpu().numpy()
    d = got - ref
    assert np.abs(ref).min() > 0.99
    assert abs(d[ref > 0].mean()) <= 3e-7 and abs(d[ref < 0].mean()) <= 3e-7
    assert np.abs(d).max() <= PEARSON_ATOL


def _offset_trend_rows(n, D, seed):
    """Grouped rows plus large per-row offsets (up to 1e4 times the spread),
    linear trends, and rows periodic with period 12, the sampling stride of
    the shift at D = 12325 (every sample falls on the same phase, so the
    shift misses the mean by the full amplitude)."""
    g = torch.Generator().manual_seed(seed)
    X = synth.vectors_grouped(n, D, seed=seed).double()
    k = torch.arange(D, dtype=torch.float64)
    off = 1e4 * (2 * torch.rand(n, 1, generator=g, dtype=torch.float64) - 1)
    off[::3] *= 1e-3
    X += off
    trend = torch.rand(n, 1, generator=g, dtype=torch.float64) * torch.linspace(-3, 3, D,
                                                                                dtype=torch.float64)
    X[1::3] += trend[1::3]
    X[2::7] += 2.0 * torch.cos(2 * np.pi * k / 12)
    return X.float().contiguous()


def test_pearson_offsets_and_trends(ap, oracle_lib):
    """Rows centred on a sampled shift in one pass: the exact mean enters as
    the correction D delta_i delta_j; every path that prepares rows (device
    and host sources, whole tiles and split-K, FP32, out-of-core macros in
    both orders, load-and-run) must match the oracle on rows whose means,
    trends and stride-aligned periods would expose a wrong correction."""
    n, D = 300, 12325
    X = _offset_trend_rows(n, D, seed=17)
    Xn = X.numpy()
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(Xn, pi, pj)
    tol = pearson_tolerance(Xn, pi, pj, 1)
    tol32 = pearson_tolerance(Xn, pi, pj, 0)

    def check(got, t, what):
        err = np.abs(got - ref)
        assert np.all(err <= t), f"{what}: max |err| {err.max():.3e}, worst {(err / t).max():.2f}x"

    both = (ap.AP_PREC_SPLIT_BF16, ap.AP_PREC_FP32)
    with ap.Items.from_vectors(X.cuda(), precisions=both) as it:
        for k in (0, -1, 3):
            it.set_plan(128, 256, 0, k)
            check(it.run_pairs().cpu().numpy(), tol, f"device k_split {k}")
        check(it.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32).cpu().numpy(), tol32, "fp32")
        assert it.last_device_error() == 0
    check(_run(ap, X, ap.AP_PREC_SPLIT_BF16, host=True), tol, "host source")
    Xp = X.pin_memory()
    cache = 3 * 256 * ((D + 63) // 64 * 64) * 4
    with ap.Items.from_vectors(Xp, slot_cache_bytes=cache) as it:
        check(it.run_pairs().cpu().numpy(), tol, "out-of-core resident+streamed")
        it.set_out_of_core_policy(ap.binding.AP_OOC_DC_LRU)
        check(it.run_pairs().cpu().numpy(), tol, "out-of-core recursive+LRU")
        it.set_out_of_core_policy(ap.binding.AP_OOC_K_SLICED)
        check(it.run_pairs().cpu().numpy(), tol, "out-of-core column slices")
        assert it.last_device_error() == 0
    with ap.Items.from_vectors(Xp) as it:
        check(it.load_and_run(Xp).cpu().numpy(), tol, "load and run")


@pytest.mark.parametrize("n,D", [(300, (1 << 19) + 77), (513, 3 * (1 << 18) + 40)])
def test_load_and_run_column_chunks(ap, oracle_lib, n, D):
    """Rows of 2 MiB and more stream in column chunks of whole 1 MiB pieces
    (here two and three, the last one ragged), centred on shifts sampled over
    the whole rows: rows with offsets, trends and periods still match the
    oracle, and the stored set gives the same correlations afterwards."""
    X = _offset_trend_rows(n, D, seed=23)
    Xn = X.numpy()
    rng = np.random.default_rng(3)
    pi, pj = oracle_lib.all_pairs(n)
    keep = rng.choice(len(pi), 1500, replace=False)
    pi, pj = pi[keep], pj[keep]
    ref = oracle_lib.pearson(Xn, pi, pj)
    tol = pearson_tolerance(Xn, pi, pj, 1)
    p = torch.from_numpy(pi.astype(np.int64) * n - pi * (pi + 1) // 2 + (pj - pi - 1)).cuda()
    Xp = X.pin_memory()
    both = (ap.AP_PREC_SPLIT_BF16, ap.AP_PREC_FP32)
    with ap.Items.from_vectors(torch.zeros(n, D, device="cuda"), precisions=both) as it:
        it.set_trace(True)
        got = it.load_and_run(Xp)
        tr = it.trace()
        st = it.stats()
        again = it.run_pairs()
        # the FP32 copy written chunk by chunk beside the split one
        got32 = it.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32)[p].cpu().numpy()
        assert it.last_device_error() == 0
    err32 = np.abs(got32 - ref)
    assert np.all(err32 <= pearson_tolerance(Xn, pi, pj, 0)), float(err32.max())
    err = np.abs(got[p].cpu().numpy() - ref)
    assert np.all(err <= tol), f"max |err| {err.max():.3e}, worst {(err / tol).max():.2f}x"
    assert np.all(np.abs(got[p].cpu().numpy() - again[p].cpu().numpy())
                  <= regroup_tolerance(Xn, pi, pj))
    assert st["h2d_bytes"] == n * D * 4
    chunks = D // (1 << 18)
    copies = [e for e in tr if e["stage"] == "copy"]
    assert len(copies) == chunks * ((n + 255) // 256)
    assert sum(e["bytes"] for e in copies) == n * D * 4
