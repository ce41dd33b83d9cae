"""Benchmark of the all-pairs hot path on GB300.

Default workload: all-pairs Pearson correlation of 8,192 FP32 vectors of
length 2^20 (i.i.d. N(0,1) noise plus a shared N(0,1) component of weight
0.05 within seeded groups of 16), split-BF16 Gram on the tensor cores with
FP64 normalisation.  One step = the whole path over the resident inputs:
pre-processing (FP64 mean / norm, centring, hi/lo split), the tiled Gram and
the Pearson epilogue into the packed upper-triangle output.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair evals/s + % of roofline; split-BF16 vs FP32 speedup at ≤1e-6 err"
N_ITEMS, DIM = 8192, 1 << 20
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one Gram launch; see
# profiles/ (None until a capture of the current kernel exists)
GRAM_TRAFFIC_BYTES = None


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return dict(FALLBACK), "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        pmax = max(r[2] for r in rows)
        load = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in load for k, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in load),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(load), "power_w_max": pmax}


def sample_rows(n, k, seed=1234):
    import numpy as np
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def run_oracle_sample(X_rows, n_threads):
    """FP64 oracle on every pair of the sampled rows; returns (pi, pj, r, seconds)."""
    import oracle
    oracle.build()
    pi, pj = oracle.all_pairs(X_rows.shape[0])
    t0 = time.perf_counter()
    mu, ss = oracle.vector_stats(X_rows, n_threads)
    r = oracle.pearson(X_rows, pi, pj, mu, ss, n_threads=n_threads)
    return pi, pj, r, time.perf_counter() - t0


def reference_arm(args):
    """The oracle as it stands, on the machine's host cores, on bounded samples."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import torch
    import synth
    cores = os.cpu_count() or 1
    k = args.ref_rows
    rows = sample_rows(N_ITEMS, k)
    # the same inputs as the GPU arm: generate on the GPU when one is present
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    if dev == "cuda":
        X = synth.vectors_grouped(N_ITEMS, DIM, seed=0, device="cuda")
        sub = X[torch.from_numpy(rows).cuda()].cpu().numpy()
        del X
        torch.cuda.empty_cache()
    else:
        sub = synth.vectors_grouped(k, DIM, seed=0).numpy()
    pairs = k * (k - 1) // 2
    for _ in range(args.warmup):
        run_oracle_sample(sub[:16], cores)
    times = []
    for _ in range(args.steps):
        times.append(run_oracle_sample(sub, cores)[3])
    t = sum(times)
    value = pairs * len(times) / t
    sample = f"all {pairs} pairs of {k} sampled vectors of the workload per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "pearson_n8192_d1048576", "n_items": N_ITEMS, "dim": DIM,
                       "sample_rows": k},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def ours(args):
    import numpy as np
    import torch
    import synth
    import paper_2009_04755_gb300 as ap

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        if ws == 1:
            return v
        import torch.distributed as dist
        t = torch.tensor([v], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    n, D = N_ITEMS, DIM
    P = n * (n - 1) // 2
    stream = torch.cuda.current_stream()
    X = synth.vectors_grouped(n, D, seed=0, device="cuda")
    items = ap.Items.from_vectors(X, precisions=(ap.AP_PREC_SPLIT_BF16,))
    out = torch.empty(P, dtype=torch.float64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 2)]

    def step(k=None):
        items.update(X)
        if k is not None:
            ev[2 * k].record(stream)
        items.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_SPLIT_BF16, out=out)
        if k is not None:
            ev[2 * k + 1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        step(k)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    ms = max_over_ranks(ms)
    gram_ms = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)]
    gram_avg = sum(gram_ms) / len(gram_ms)
    value = P * ws * args.steps / (ms / 1e3)
    if items.last_device_error() != 0:
        raise RuntimeError("device wait timed out during the benchmark")

    pk, pk_kind = peaks()
    peak_tf = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    flops_launch = 3 * 2.0 * D * P          # three BF16 products per pair, 2 flops per MAC
    achieved_tf = flops_launch / (gram_avg / 1e3) / 1e12
    traffic = None if GRAM_TRAFFIC_BYTES is None else GRAM_TRAFFIC_BYTES
    roofline = {"bound": "tensor", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved_tf / peak_tf, "traffic": traffic,
                "kernel": "gram_tc_kernel", "peak_kind": f"{pk_kind} bf16 sustained",
                "algorithmic_flops_per_launch": flops_launch}

    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3/fp32-acc/fp64-norm", "data": "synthetic",
            "config": {"workload": "pearson_n8192_d1048576", "n_items": n, "dim": D,
                       "pairs": P, "precision": "split-bf16",
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs (32 GiB raw + 32 GiB hi/lo) far larger than L2"},
            "roofline": roofline, "gram_ms": gram_avg,
            "gpu_launches": 3 * args.steps}
    if clk:
        line["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}

    # ---- FP32 CUDA-core comparator (same launch shape, Gram + epilogue) ----
    if not args.no_fp32:
        items32 = ap.Items.from_vectors(X, precisions=(ap.AP_PREC_FP32,))
        out32 = torch.empty(P, dtype=torch.float64, device="cuda")
        items32.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32, out=out32)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        items32.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32, out=out32)
        e1.record(stream)
        torch.cuda.synchronize()
        items32.close()
        f32_ms = e0.elapsed_time(e1)
        line["fp32_gram_ms"] = f32_ms
        line["split_vs_fp32_speedup"] = f32_ms / gram_avg
    else:
        out32 = None

    # ---- the oracle on a bounded sample: CPU baseline and error check ----
    if rank == 0 and not args.no_cpu:
        k = args.ref_rows
        rows = sample_rows(n, k)
        sub = X[torch.from_numpy(rows).cuda()].cpu().numpy()
        cores = os.cpu_count() or 1
        pi, pj, r_ref, secs = run_oracle_sample(sub, cores)
        gi, gj = rows[pi], rows[pj]
        p = torch.from_numpy(gi * n - gi * (gi + 1) // 2 + (gj - gi - 1)).cuda()
        err = float(np.abs(out[p].cpu().numpy() - r_ref).max())
        line["max_abs_err_sampled"] = {"split_bf16": err}
        if out32 is not None:
            line["max_abs_err_sampled"]["fp32"] = float(
                np.abs(out32[p].cpu().numpy() - r_ref).max())
        line["cpu_baseline"] = {"value": len(pi) / secs, "unit": "pairs/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"all {len(pi)} pairs of {k} sampled vectors "
                                          f"(FP64 two-pass stats + centred sums)"}

    # ---- end to end through the C ABI from pinned host memory ----
    if not args.no_e2e:
        del X
        torch.cuda.empty_cache()
        Xh = synth.vectors_grouped(n, D, seed=0, device="cuda").cpu().pin_memory()
        res_h = torch.empty(P, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        items.update(Xh)                     # warm the host path once
        items.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_SPLIT_BF16, out=out)
        res_h.copy_(out, non_blocking=True)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ksteps = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(ksteps):
            items.update(Xh)
            items.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_SPLIT_BF16, out=out)
            res_h.copy_(out, non_blocking=True)
        e1.record(stream)
        barrier()
        e_ms = max_over_ranks(e0.elapsed_time(e1))
        line["e2e"] = {"value": P * ws * ksteps / (e_ms / 1e3), "unit": "pairs/s",
                       "h2d_bytes_per_step": int(n * D * 4),
                       "d2h_bytes_per_step": int(P * 8), "steps": ksteps,
                       "ms_per_step": e_ms / ksteps}
    items.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-rows", type=int, default=512,
                    help="vectors in the oracle's bounded sample (all their pairs)")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
