"""GPU parity of the pair-list entry points (the pair function on a chosen
subset of pairs) against the FP64 oracle, and against the all-pairs run:
a pair listed in packed order goes through the same operations, so its
result has the same bits."""
import numpy as np
import pytest

import synth
from gpu_util import (PEARSON_ATOL, check_grad, check_overlap, cloud_wsum, pearson_tolerance)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ap():
    import paper_2009_04755_gb300 as ap
    ap.lib()
    return ap


def _random_list(n, m, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n, m)
    b = rng.integers(0, n, m)
    b = np.where(a == b, (b + 1) % n, b)
    return a.astype(np.int32), b.astype(np.int32)


def _packed(pi, pj, n):
    i, j = np.minimum(pi, pj).astype(np.int64), np.maximum(pi, pj).astype(np.int64)
    return i * n - i * (i + 1) // 2 + (j - i - 1)


@pytest.mark.parametrize("dim", [2, 3])
def test_overlap_list_matches_oracle_and_all_pairs(ap, oracle_lib, dim):
    if dim == 2:
        c = synth.clouds_uniform(n=120, dim=2, size=(20, 300), seed=3)
    else:   # uneven sizes: stored sorted by size, listed by original id
        c = synth.clouds_lognormal(n=90, dim=3, median=200, clip=(20, 2500), seed=4)
    n = len(c["offsets"]) - 1
    pi, pj = _random_list(n, 700, seed=dim)
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, with_cond=True)
    with ap.Items.from_clouds(c) as it:
        got = it.run_pairs_list(pi, pj).cpu().numpy()
        full = it.run_pairs().cpu().numpy()
        assert it.last_device_error() == 0
    check_overlap(got, ref, kappa, bound, f"list {dim}d")
    if dim == 2:   # stored in item order: a pair listed as (a < b) has the same bits
        fwd = pi < pj
        np.testing.assert_array_equal(got[fwd], full[_packed(pi, pj, n)[fwd]])
    else:          # sorted storage: the roles of a and b may differ, not the value
        np.testing.assert_allclose(got, full[_packed(pi, pj, n)], rtol=2e-5, atol=1e-30)


def test_overlap_list_transform_on_second_item(ap, oracle_lib):
    c = synth.clouds_templates(n=48, seed=5)
    pi, pj = _random_list(48, 400, seed=9)
    rng = np.random.default_rng(1)
    params = np.stack([rng.uniform(-np.pi, np.pi, 400), rng.uniform(-0.3, 0.3, 400),
                       rng.uniform(-0.3, 0.3, 400)], 1).astype(np.float32)
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, params=params.astype(np.float64),
                                           with_cond=True)
    with ap.Items.from_clouds(c) as it:
        got = it.run_pairs_list(pi, pj, params=torch.from_numpy(params).cuda()).cpu().numpy()
    check_overlap(got, ref, kappa, bound, "list with transforms")


@pytest.mark.parametrize("fn", ["l2", "bc"])
def test_score_list(ap, oracle_lib, fn):
    c = synth.clouds_uniform(n=64, dim=2, size=(50, 200), seed=12)
    pi, pj = _random_list(64, 300, seed=13)
    f = ap.AP_FN_GMM_L2 if fn == "l2" else ap.AP_FN_BHATTACHARYYA
    with ap.Items.from_clouds(c) as it:
        got = it.run_pairs_list(pi, pj, fn=f).cpu().numpy()
        full = it.run_pairs(f).cpu().numpy()
    fwd = pi < pj
    np.testing.assert_array_equal(got[fwd], full[_packed(pi, pj, 64)[fwd]])
    if fn == "l2":
        ref, bd = oracle_lib.gmm_l2(c, pi, pj, with_bound=True)
        S = oracle_lib.gmm_self(c)
        mag = S[pi] + S[pj] + np.abs(S[pi] + S[pj] - ref)
    else:
        ref, bd = oracle_lib.bhattacharyya(c, pi, pj, with_bound=True)
        mag = np.abs(ref)
    assert np.all(np.abs(got - ref) <= 4 * bd + 4e-6 * mag + 1e-30)


def test_backward_and_ascent_list(ap, oracle_lib):
    c = synth.clouds_templates(n=40, seed=7)
    pi, pj = _random_list(40, 250, seed=21)
    rng = np.random.default_rng(3)
    params = np.stack([rng.uniform(-0.2, 0.2, 250), rng.uniform(-0.05, 0.05, 250),
                       rng.uniform(-0.05, 0.05, 250)], 1).astype(np.float32)
    f_ref, g_ref = oracle_lib.overlap_grad(c, pi, pj, params=params.astype(np.float64))
    with ap.Items.from_clouds(c) as it:
        g, f = it.backward_list(pi, pj, params=torch.from_numpy(params).cuda())
        check_grad(g.cpu().numpy(), g_ref, cloud_wsum(c, pi, pj))
        # one ascent step = the oracle's step from the same parameters
        prm = torch.from_numpy(params.copy()).cuda()
        it.ascent_list(pi, pj, prm, 1, 1e-3)
        new_ref, _, _, _ = oracle_lib.ascent_step(c, pi, pj, params.astype(np.float64), 1e-3)
        step = new_ref - params
        got_step = prm.cpu().numpy().astype(np.float64) - params
        assert np.all(np.abs(got_step - step) <= 1e-4 * np.abs(step).max(1, keepdims=True) + 1e-9)
        # pairs in packed order: the list's ascent = the all-pairs ascent there
        fwd = np.flatnonzero(pi < pj)
        keep = fwd[np.unique(_packed(pi, pj, 40)[fwd], return_index=True)[1]]
        P = 40 * 39 // 2
        full = torch.zeros(P, 3, device="cuda")
        sub = torch.zeros(len(keep), 3, device="cuda")
        it.ascent(full, 5, 1e-3)
        it.ascent_list(pi[keep], pj[keep], sub, 5, 1e-3)
        np.testing.assert_array_equal(sub.cpu().numpy(),
                                      full.cpu().numpy()[_packed(pi[keep], pj[keep], 40)])
        assert it.last_device_error() == 0


def test_autograd_list(ap, oracle_lib):
    from paper_2009_04755_gb300.autograd import overlap_align_list
    c = synth.clouds_templates(n=30, seed=6)
    pi, pj = _random_list(30, 120, seed=8)
    rng = np.random.default_rng(4)
    prm = np.stack([rng.uniform(-0.3, 0.3, 120), rng.uniform(-0.05, 0.05, 120),
                    rng.uniform(-0.05, 0.05, 120)], 1).astype(np.float32)
    w = rng.uniform(0.5, 1.5, 120)
    f_ref, g_ref = oracle_lib.overlap_grad(c, pi, pj, prm.astype(np.float64))
    with ap.Items.from_clouds(c) as it:
        p = torch.from_numpy(prm).cuda().requires_grad_(True)
        f = overlap_align_list(it, pi, pj, p)
        (f * torch.from_numpy(w).float().cuda()).sum().backward()
        grad = p.grad.cpu().numpy()
    check_grad(grad, g_ref * w[:, None], cloud_wsum(c, pi, pj) * w)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("m,D", [(2000, 12325), (40, 12325), (500, 50)])
def test_pearson_list(ap, oracle_lib, prec, m, D):
    """2000 pairs over three row blocks read a row-major copy of the rows
    (the last 128-column group holds 64, the last block 44 rows); 40 pairs
    read the blocked arrays in place; rows of 50 values are one 64-column
    group of the copy."""
    n = 300
    X = synth.vectors_grouped(n, D, seed=31) + torch.linspace(-5, 5, n)[:, None]
    X = X.contiguous()
    pi, pj = _random_list(n, m, seed=prec)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    with ap.Items.from_vectors(X.cuda(), precisions=(prec,)) as it:
        got = it.run_pairs_list(pi, pj, ap.AP_FN_PEARSON, prec).cpu().numpy()
        assert it.last_device_error() == 0
    tol = pearson_tolerance(X.numpy(), pi, pj, prec)
    assert np.all(np.abs(got - ref) <= tol), float(np.abs(got - ref).max())


def test_pearson_list_full_size_rows(ap, oracle_lib):
    """Rows of the benchmark's length (2^20): the list path at 1e-6."""
    n, D = 64, 1 << 20
    X = synth.vectors_grouped(n, D, seed=2)
    pi, pj = _random_list(n, 200, seed=5)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    with ap.Items.from_vectors(X.cuda()) as it:
        got = it.run_pairs_list(pi, pj).cpu().numpy()
    assert np.abs(got - ref).max() <= PEARSON_ATOL


def test_cosine_list(ap, oracle_lib):
    off, idx, val = synth.sparse_cv(60, dim=200000, nnz=(20, 20000), common=3000, seed=8)
    # rows of every size; row 7 emptied (its pairs are NaN)
    rows = [idx[off[k]:off[k + 1]] for k in range(60)]
    rows[7] = rows[7][:0]
    vals = [val[off[k]:off[k + 1]] for k in range(60)]
    vals[7] = vals[7][:0]
    off2 = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    idx2, val2 = np.concatenate(rows), np.concatenate(vals)
    pi, pj = _random_list(60, 500, seed=4)
    pi[:5], pj[:5] = 7, np.arange(5)                  # the empty row: NaN
    ref = oracle_lib.sparse_cosine(off2, idx2, val2, pi, pj)
    with ap.Items.from_sparse(off2, idx2, val2, 200000) as it:
        got = it.run_pairs_list(pi, pj).cpu().numpy()
        full = it.run_pairs().cpu().numpy()
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan) and nan[:5].all()
    mag = oracle_lib.sparse_cosine(off2, idx2, np.abs(val2), pi, pj)
    tol = 2.0 ** -20 * np.nan_to_num(mag) + 1e-12
    assert np.all(np.abs(got[~nan] - ref[~nan]) <= tol[~nan])
    good = ~nan
    np.testing.assert_allclose(got[good], full[_packed(pi, pj, 60)][good], rtol=0, atol=1e-6)


def test_list_rejects_bad_pairs(ap):
    c = synth.clouds_uniform(n=10, dim=2, size=(5, 9), seed=1)
    with ap.Items.from_clouds(c) as it:
        for a, b in [([0], [0]), ([0], [10]), ([-1], [2])]:
            with pytest.raises(ap.APError):
                it.run_pairs_list(a, b)
        with pytest.raises(ap.APError):                       # a vector function
            it.run_pairs_list([0], [1], fn=ap.AP_FN_PEARSON)
        assert it.run_pairs_list([], []).numel() == 0
    X = torch.randn(8, 64)
    with ap.Items.from_vectors(X.cuda()) as it:
        with pytest.raises(ap.APError) as e:                  # FP32 copy not built
            it.run_pairs_list([0], [1], ap.AP_FN_PEARSON, ap.AP_PREC_FP32)
        assert e.value.status == 6
        with pytest.raises(ap.APError):
            it.ascent_list([0], [1], torch.zeros(1, 3, device="cuda"), 1, 1e-3)
