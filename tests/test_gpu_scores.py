"""GPU parity of the two particle scores (Sec. V-C): the squared L2 distance
between Gaussian mixtures and the Bhattacharyya cost, against the FP64 oracle,
through the C ABI."""
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


def _gpu(ap, c, fn, params=None, twice=False):
    with ap.Items.from_clouds(c) as it:
        prm = None if params is None else torch.as_tensor(params, dtype=torch.float32).cuda()
        out = it.run_pairs(fn, params=prm).cpu().numpy()
        if twice:                                  # the cached storage and graph
            again = it.run_pairs(fn, params=prm).cpu().numpy()
            np.testing.assert_array_equal(again, out)
        assert it.last_device_error() == 0
    return out


def _check(oracle_lib, c, pi, pj, got, which, params=None):
    """|gpu - oracle| <= 4 x the oracle's FP32 error scale of the terms (each
    exponent, reciprocal square root and power carries a few 2^-23 of its
    term) + 4e-6 of the summed term magnitudes (FP32 partial sums of up to 64
    terms before they reach FP64)."""
    prm = None if params is None else params.astype(np.float64)
    if which == "l2":
        ref, bound = oracle_lib.gmm_l2(c, pi, pj, params=prm, with_bound=True)
        S = oracle_lib.gmm_self(c)
        cross = (S[pi] + S[pj] - ref) / 2
        mag = S[pi] + S[pj] + 2 * np.abs(cross)
    else:
        ref, bound = oracle_lib.bhattacharyya(c, pi, pj, params=prm, with_bound=True)
        mag = np.abs(ref)
    err = np.abs(got.astype(np.float64) - ref)
    lim = 4 * bound + 4e-6 * mag + 1e-30
    bad = err > lim
    assert not bad.any(), f"{which}: {bad.sum()} pairs over, worst {(err / lim).max():.2f}x"
    return float((err / np.maximum(mag, 1e-30)).max())


@pytest.mark.parametrize("fn", ["l2", "bc"])
def test_scores_2d_all_pairs(ap, oracle_lib, fn):
    c = synth.clouds_uniform(n=96, dim=2, size=(64, 160), seed=11)
    pi, pj = oracle_lib.all_pairs(96)
    f = ap.AP_FN_GMM_L2 if fn == "l2" else ap.AP_FN_BHATTACHARYYA
    _check(oracle_lib, c, pi, pj, _gpu(ap, c, f, twice=True), fn)


@pytest.mark.parametrize("fn", ["l2", "bc"])
def test_scores_3d_lognormal(ap, oracle_lib, fn):
    # uneven sizes: the sorted plan, items above one chunk of a row job
    c = synth.clouds_lognormal(n=60, dim=3, median=300, clip=(50, 2500), seed=9)
    pi, pj = oracle_lib.all_pairs(60)
    f = ap.AP_FN_GMM_L2 if fn == "l2" else ap.AP_FN_BHATTACHARYYA
    _check(oracle_lib, c, pi, pj, _gpu(ap, c, f), fn)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fn", ["l2", "bc"])
def test_scores_weights_and_ragged(ap, oracle_lib, dim, fn):
    rng = np.random.default_rng(20 + dim)
    sizes = np.array([0, 1, 3, 64, 65, 129, 0, 7, 300, 2])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    tot = int(off[-1])
    pts = rng.uniform(-0.2, 0.2, (tot, 3)).astype(np.float32)
    c = {"dim": dim, "offsets": off, "x": pts[:, 0].copy(), "y": pts[:, 1].copy(),
         "z": pts[:, 2].copy() if dim == 3 else None,
         "sigma": rng.uniform(0.02, 0.08, tot).astype(np.float32),
         "weight": rng.uniform(0.0, 2.0, tot).astype(np.float32)}
    c["weight"][::7] = 0.0
    n = len(sizes)
    pi, pj = oracle_lib.all_pairs(n)
    f = ap.AP_FN_GMM_L2 if fn == "l2" else ap.AP_FN_BHATTACHARYYA
    got = _gpu(ap, c, f)
    _check(oracle_lib, c, pi, pj, got, fn)
    if fn == "bc":
        empty = (sizes[pi] == 0) | (sizes[pj] == 0)
        assert np.all(got[empty] == 0.0)


@pytest.mark.parametrize("fn", ["l2", "bc"])
def test_scores_with_transform(ap, oracle_lib, fn):
    c = synth.clouds_templates(n=32, seed=6)
    pi, pj = oracle_lib.all_pairs(32)
    rng = np.random.default_rng(2)
    params = np.stack([rng.uniform(-np.pi, np.pi, len(pi)), rng.uniform(-0.3, 0.3, len(pi)),
                       rng.uniform(-0.3, 0.3, len(pi))], 1).astype(np.float32)
    f = ap.AP_FN_GMM_L2 if fn == "l2" else ap.AP_FN_BHATTACHARYYA
    _check(oracle_lib, c, pi, pj, _gpu(ap, c, f, params), fn, params)


def test_l2_distance_of_identical_items_is_small(ap, oracle_lib):
    """Two copies of one particle: the distance is a cancellation of S_i +
    S_j - 2C down to the FP32 error of the terms."""
    c = synth.clouds_uniform(n=1, dim=2, size=(300, 300), seed=4)
    two = {k: (np.concatenate([v, v]) if isinstance(v, np.ndarray) and k != "offsets" else v)
           for k, v in c.items()}
    two["offsets"] = np.array([0, 300, 600], np.int64)
    got = _gpu(ap, two, ap.AP_FN_GMM_L2)
    S = oracle_lib.gmm_self(two)
    assert abs(float(got[0])) <= 1e-5 * S[0]
