"""Failure detection without a GPU fault: a bounded device wait is made to
run out (the producer withholds a stage nothing else will fill), the kernel
records its status and leaves cleanly, the host reads the code, and the
context keeps working for the next launch.  The withheld stage is either the
first of each tile (no tensor-core MMA issued yet) or a later one (MMAs of the
tile issued and not yet committed to an accumulator barrier when the wait
runs out: they must be drained before TMEM is freed)."""
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


def test_wait_runs_out_and_context_survives(ap, oracle_lib):
    n, D = 300, 2048
    X = synth.vectors_grouped(n, D, seed=8)
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    with ap.Items.from_vectors(X.cuda()) as it:
        it.set_debug(1, wait_budget_ns=50_000_000)      # 50 ms per wait
        it.run_pairs()
        torch.cuda.synchronize()                          # returns: nothing hangs
        code = it.last_device_error()
        assert code in (1, 2, 3)                          # a wait ran out and said so
        assert it.last_device_error() == 0                # reading clears it
        it.set_debug(0, 0)
        got = it.run_pairs().cpu().numpy()                # the context still works
        assert it.last_device_error() == 0
    assert np.abs(got - ref).max() < 1e-4


@pytest.mark.parametrize("k_split", [-1, 0])
def test_wait_runs_out_with_mmas_in_flight(ap, oracle_lib, k_split):
    # k_split -1: the default split-K units (two k-blocks each here, the
    # second withheld); 0: whole tiles of 64 k-blocks, the sixth withheld,
    # inside the first seeded 256-column chain
    n, D = 300, 2048
    X = synth.vectors_grouped(n, D, seed=9)
    pi, pj = oracle_lib.all_pairs(n)
    ref = oracle_lib.pearson(X.numpy(), pi, pj)
    with ap.Items.from_vectors(X.cuda()) as it:
        it.set_plan(128, 256, 0, k_split)
        for _ in range(2):                                # twice: nothing is left behind
            it.set_debug(2, wait_budget_ns=50_000_000)
            it.run_pairs()
            torch.cuda.synchronize()
            assert it.last_device_error() in (1, 2, 3)
            it.set_debug(0, 0)
            got = it.run_pairs().cpu().numpy()
            assert it.last_device_error() == 0
            assert np.abs(got - ref).max() < 1e-4


def test_set_debug_rejects_unknown_flag(ap):
    X = torch.randn(10, 64, device="cuda")
    with ap.Items.from_vectors(X) as it:
        with pytest.raises(ap.APError):
            it.set_debug(7)
