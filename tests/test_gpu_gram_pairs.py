"""The split-BF16 Gram on CTA pairs (tcgen05.mma.cta_group::2, 256 x 256
block pairs over two SMs) against the FP64 oracle, the single-CTA kernel and
bit-exact pair coverage, through the C ABI: both kernels, split-K units in
waves and whole block pairs, ragged item counts (a pair's second CTA or the
J block's second half past the last item) and short, odd-length vectors."""
import numpy as np
import pytest

import synth
from gpu_util import pearson_tolerance, regroup_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ap():
    import paper_2009_04755_gb300 as ap
    ap.lib()
    return ap


def _pearson(ap, X, k_split, mma_ctas):
    with ap.Items.from_vectors(X.cuda()) as it:
        it.set_plan(128, 256, 0, k_split, mma_ctas)
        plan = it.plan()
        assert plan["mma_ctas"] == mma_ctas
        out = it.run_pairs().cpu().numpy()
        assert it.last_device_error() == 0
    return out


@pytest.mark.parametrize("n,D", [(300, 2048), (513, 4160), (1000, 1000), (129, 64)])
@pytest.mark.parametrize("k_split", [-1, 0, 3])
@pytest.mark.parametrize("mma_ctas", [1, 2])
def test_gram_kernels_match_oracle(ap, oracle_lib, n, D, k_split, mma_ctas):
    X = synth.vectors_grouped(n, D, seed=7 * n + D)
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    got = _pearson(ap, X, k_split, mma_ctas)
    tol = pearson_tolerance(X.numpy(), pi, pj, 1)
    over = np.abs(got - ref) > tol
    assert not over.any(), f"{over.sum()} pairs beyond tolerance, max |err| " \
        f"{np.abs(got - ref).max():.3e}"


@pytest.mark.parametrize("n,D", [(300, 2048), (1000, 8192)])
def test_pair_kernel_agrees_with_single_cta_kernel(ap, oracle_lib, n, D):
    # the same products chained the same way: agreement to rounding of the
    # accumulation, far inside the regrouping allowance
    X = synth.vectors_grouped(n, D, seed=n + 5)
    pi, pj = oracle_lib.all_pairs(n)
    for k_split in (-1, 0):
        a = _pearson(ap, X, k_split, 1)
        b = _pearson(ap, X, k_split, 2)
        assert np.all(np.abs(a - b) <= regroup_tolerance(X.numpy(), pi, pj))


@pytest.mark.parametrize("n", [2, 255, 257, 777, 1024])
def test_pair_kernel_coverage_every_pair_once(ap, oracle_lib, n):
    X = synth.vectors_grouped(n, 64, seed=n)
    with ap.Items.from_vectors(X.cuda()) as it:
        it.set_plan(128, 256, 0, -1, 2)
        cnt = it.run_pairs(ap.AP_FN_COVERAGE).cpu().numpy()
    assert cnt.shape == (oracle_lib.pair_count(n),)
    assert np.all(cnt == 1)


def test_set_plan_rejects_bad_mma_ctas(ap):
    X = torch.randn(10, 64)
    with ap.Items.from_vectors(X.cuda()) as it:
        with pytest.raises(ap.APError):
            it.set_plan(128, 256, 0, -1, 3)
        assert it.plan()["mma_ctas"] == 2          # the default
