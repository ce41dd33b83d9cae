"""GPU parity of the Gaussian overlap cost (2-D and 3-D point clouds) against
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from gpu_util import check_overlap

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ap():
    import paper_2009_04755_gb300 as ap
    ap.lib()
    return ap


def _gpu_overlap(ap, c, params=None):
    with ap.Items.from_clouds(c) as it:
        prm = None if params is None else torch.as_tensor(params, dtype=torch.float32).cuda()
        f = it.run_pairs(ap.AP_FN_OVERLAP, params=prm).cpu().numpy()
        assert it.last_device_error() == 0
    return f


def test_overlap_2d_n256_all_pairs(ap, oracle_lib):
    """256 2-D clouds of 64-128 points, every one of the 32,640 pairs."""
    c = synth.clouds_uniform(n=256, dim=2, size=(64, 128), seed=0)
    pi, pj = oracle_lib.all_pairs(256)
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, with_cond=True)
    f = _gpu_overlap(ap, c)
    assert f.shape == ref.shape
    check_overlap(f, ref, kappa, bound, "2d n256")


def test_overlap_3d_lognormal_sorted(ap, oracle_lib):
    # uneven sizes take the size-sorted plan; includes items far above one chunk
    c = synth.clouds_lognormal(n=160, dim=3, median=300, clip=(50, 3000), seed=5)
    pi, pj = oracle_lib.all_pairs(160)
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, with_cond=True)
    check_overlap(_gpu_overlap(ap, c), ref, kappa, bound, "3d lognormal")


@pytest.mark.parametrize("dim", [2, 3])
def test_overlap_weights_and_ragged(ap, oracle_lib, dim):
    rng = np.random.default_rng(dim)
    sizes = np.array([0, 1, 3, 4, 5, 33, 64, 65, 127, 128, 129, 200, 0, 7, 300, 2])
    c = synth.clouds_uniform(n=len(sizes), dim=dim, size=(1, 2), seed=dim)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    tot = int(off[-1])
    pts = rng.uniform(-0.3, 0.3, (tot, 3)).astype(np.float32)
    c = {"dim": dim, "offsets": off, "x": pts[:, 0].copy(), "y": pts[:, 1].copy(),
         "z": pts[:, 2].copy() if dim == 3 else None,
         "sigma": rng.uniform(0.02, 0.08, tot).astype(np.float32),
         "weight": rng.uniform(0.0, 2.0, tot).astype(np.float32)}
    c["weight"][::7] = 0.0
    n = len(sizes)
    pi, pj = oracle_lib.all_pairs(n)
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, with_cond=True)
    f = _gpu_overlap(ap, c)
    # empty items give exactly 0
    empty = (sizes[pi] == 0) | (sizes[pj] == 0)
    assert np.all(f[empty] == 0.0)
    check_overlap(f[~empty], ref[~empty], kappa[~empty], bound[~empty], f"ragged {dim}d")


def test_overlap_with_transform(ap, oracle_lib):
    c = synth.clouds_templates(n=40, seed=4)
    pi, pj = oracle_lib.all_pairs(40)
    rng = np.random.default_rng(1)
    params = np.stack([rng.uniform(-np.pi, np.pi, len(pi)), rng.uniform(-0.3, 0.3, len(pi)),
                       rng.uniform(-0.3, 0.3, len(pi))], 1).astype(np.float32)
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, params=params.astype(np.float64),
                                           with_cond=True)
    check_overlap(_gpu_overlap(ap, c, params), ref, kappa, bound, "transform")


@pytest.mark.parametrize("dim,n", [(2, 256), (3, 500), (2, 3)])
def test_overlap_coverage_every_pair_once(ap, dim, n):
    c = (synth.clouds_lognormal(n=n, dim=3, clip=(50, 2000), seed=1) if dim == 3
         else synth.clouds_uniform(n=n, dim=2, seed=1))
    with ap.Items.from_clouds(c) as it:
        cnt = it.run_pairs(ap.AP_FN_COVERAGE).cpu().numpy()
    assert cnt.shape == (n * (n - 1) // 2,)
    assert np.all(cnt == 1)


def test_overlap_small_n(ap):
    for n in (0, 1):
        c = synth.clouds_uniform(n=max(n, 1), dim=2, seed=0)
        c["offsets"] = c["offsets"][:n + 1]
        with ap.Items.from_clouds(c) as it:
            assert it.run_pairs().numel() == 0


def test_overlap_symmetric_at_identity(ap):
    # f(i, j) computed with the roles swapped (reverse the item order)
    c = synth.clouds_uniform(n=30, dim=2, seed=3)
    f = _gpu_overlap(ap, c)
    n = 30
    off = c["offsets"]
    order = np.arange(n)[::-1]
    sizes = np.diff(off)[order]
    roff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    idx = np.concatenate([np.arange(off[k], off[k + 1]) for k in order])
    rc = {"dim": 2, "offsets": roff, "x": c["x"][idx], "y": c["y"][idx], "z": None,
          "sigma": c["sigma"][idx], "weight": c["weight"][idx]}
    g = _gpu_overlap(ap, rc)
    for i, j in [(0, 1), (3, 17), (28, 29), (0, 29)]:
        p = ap.pair_index(i, j, n)
        q = ap.pair_index(n - 1 - j, n - 1 - i, n)
        assert abs(f[p] - g[q]) <= 1e-5 * abs(f[p])


def test_clouds_created_on_a_side_stream_from_pinned_host(ap, oracle_lib):
    # creation copies and packs on the caller's stream: the pairs run on the
    # same stream with no host synchronisation in between
    c = synth.clouds_uniform(n=40, dim=2, size=(20, 60), seed=12)
    pi, pj = oracle_lib.all_pairs(40)
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, with_cond=True)
    s = torch.cuda.Stream()
    it = ap.Items.from_clouds(c, device="cpu", stream=s, sync=False)
    out = it.run_pairs(stream=s)
    s.synchronize()
    check_overlap(out.cpu().numpy(), ref, kappa, bound, "side stream")
    it.close()
