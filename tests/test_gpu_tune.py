"""GPU checks of the tile-plan autotuner and of CUDA-graph replay: any plan
the tuner can pick gives results within tolerance of the oracle, replays are
bit-identical to direct launches, and explicit plans round-trip."""
import numpy as np
import pytest

import synth
from gpu_util import check_grad, check_overlap, cloud_wsum

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ap():
    import paper_2009_04755_gb300 as ap
    ap.lib()
    return ap


def test_tune_then_parity_2d(ap, oracle_lib):
    c = synth.clouds_uniform(n=256, dim=2, size=(64, 128), seed=0)
    pi, pj = oracle_lib.all_pairs(256)
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, with_cond=True)
    with ap.Items.from_clouds(c) as it:
        plan = it.tune(0)
        assert plan["rate"] > 0
        assert plan["block_items"] in (2, 4, 8, 16, 32)
        assert plan["block_pts"] in (2048, 4096, 8192)
        assert plan["reg_r"] in (2, 4)
        assert it.plan()["block_items"] == plan["block_items"]
        f1 = it.run_pairs().cpu().numpy()
        f2 = it.run_pairs().cpu().numpy()          # replayed from the cached graph
    check_overlap(f1, ref, kappa, bound, "tuned 2d")
    assert np.array_equal(f1, f2)


@pytest.mark.parametrize("bi,bp,rr", [(2, 2048, 2), (32, 8192, 4), (5, 100, 2), (1, 64, 4)])
def test_every_plan_is_correct_3d(ap, oracle_lib, bi, bp, rr):
    c = synth.clouds_lognormal(n=120, dim=3, median=200, clip=(50, 1500), seed=9)
    pi, pj = oracle_lib.all_pairs(120)
    ref, kappa, bound = oracle_lib.overlap(c, pi, pj, with_cond=True)
    with ap.Items.from_clouds(c) as it:
        it.set_plan(bi, bp, rr)
        f = it.run_pairs().cpu().numpy()
        cnt = it.run_pairs(ap.AP_FN_COVERAGE).cpu().numpy()
    check_overlap(f, ref, kappa, bound, f"plan {bi}/{bp}/{rr}")
    assert np.all(cnt == 1)


def test_set_plan_rejects(ap):
    c = synth.clouds_uniform(n=20, dim=2, seed=1)
    with ap.Items.from_clouds(c) as it:
        for bad in [(0, 4096, 2), (33, 4096, 2), (4, 32, 2), (4, 9000, 2), (4, 4096, 3), (4, 4096, 1)]:
            with pytest.raises(ap.APError):
                it.set_plan(*bad)


def test_tune_adjoint_then_ascent(ap, oracle_lib):
    n = 40
    c = synth.clouds_templates(n=n, seed=21)
    pi, pj = oracle_lib.all_pairs(n)
    with ap.Items.from_clouds(c) as it:
        plan = it.tune(1)
        assert plan["rate"] > 0
        g, f = it.backward(params=None)
        p = torch.zeros(len(pi), 3, device="cuda")
        p1, f1, _ = it.ascent(p.clone(), 4, 1e-3)
        p2, f2, _ = it.ascent(p.clone(), 4, 1e-3)   # second call replays the graph
        assert torch.equal(p1, p2) and torch.equal(f1, f2)
    f_ref, g_ref = oracle_lib.overlap_grad(c, pi, pj, None)
    check_grad(g.cpu().numpy(), g_ref, cloud_wsum(c, pi, pj))


def test_graph_replay_respects_new_buffers(ap):
    c = synth.clouds_uniform(n=64, dim=2, seed=2)
    with ap.Items.from_clouds(c) as it:
        a = it.run_pairs().clone()
        out = torch.zeros_like(a)
        it.run_pairs(out=out)                     # a new output buffer: a new graph
        assert torch.equal(a, out)
        it.set_plan(4, 2048, 4)                   # a new plan invalidates the graphs
        b = it.run_pairs()
        assert torch.allclose(a, b, rtol=1e-5, atol=0)
