"""The N > 1 path on CPU: two gloo ranks run the benchmark's rank plumbing
(barrier, max over ranks, whole-job rate) around independent replicas of a
small workload, as `torchrun --nproc-per-node 2 bench.py --gpus 2` does on
GPUs with NCCL.  Each replica's result must match a single-process run and
the reported rate must be the units of both ranks over the slower one."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import time

    import bench
    import oracle
    import synth
    ranks = bench.Ranks("gloo", "cpu")
    n, D, steps = 24, 512, 2
    X = synth.vectors_grouped(n, D, seed=rank).numpy()     # one replica per rank
    pi, pj = oracle.all_pairs(n)
    ranks.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        r = oracle.pearson(X, pi, pj, n_threads=1)
    ms = (time.perf_counter() - t0) * 1e3
    ranks.barrier()
    max_ms = ranks.max_over_ranks(ms)
    q.put((rank, ms, max_ms, ranks.job_rate(len(pi), steps, max_ms), r))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_job_rate(oracle_lib):
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, max0, rate0, out0), (r1, ms1, max1, rate1, out1) = res
    assert max0 == max1 == max(ms0, ms1)
    n_pairs = 24 * 23 // 2
    assert rate0 == rate1 == pytest.approx(n_pairs * 2 * 2 / (max0 / 1e3))
    for rank, out in ((0, out0), (1, out1)):
        X = synth.vectors_grouped(24, 512, seed=rank).numpy()
        pi, pj = oracle_lib.all_pairs(24)
        np.testing.assert_array_equal(out, oracle_lib.pearson(X, pi, pj, n_threads=1))


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle and prints; the others
    leave without work."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        ref_rows, steps, warmup = 8, 1, 0
    assert bench.reference_arm(Args()) == 0
    assert capsys.readouterr().out == ""
