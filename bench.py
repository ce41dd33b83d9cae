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
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one Gram launch at
# 8192 x 2^20 with its default schedule (64 column ranges of 16384 columns per
# block pair, in waves of one block pair per CTA or CTA pair), per kernel as
# it stands; None whenever the kernel has changed since the capture.
#   gram_tc_kernel: captured at full size (a one-pass metric set).
#   gram_tc2_kernel: captured at 8192 x 65536 (11,145,696,768 read +
#     1,043,277,824 written), whose schedule is the same waves with 4 ranges
#     instead of 64: every range of a wave reads and adds the same amount, so
#     the full launch moves 16 times as much.
GRAM_TRAFFIC_BYTES = {"gram_tc_kernel": 305428372992 + 17525829632,
                      "gram_tc2_kernel": 16 * (11145696768 + 1043277824)}


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


class Ranks:
    """The multi-rank plumbing of a run: one process per GPU (torchrun), each
    rank an independent replica of the workload (weak scaling, no collective
    on the data path); the only collectives are the barrier around the timed
    region and the max over ranks of its time."""

    def __init__(self, backend: str = "nccl", device: str = "cuda"):
        self.ws, self.rank, self.local = dist_env()
        self.device = device
        if self.ws > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group(backend)

    def barrier(self):
        import torch
        if self.ws > 1:
            import torch.distributed as dist
            dist.barrier()
        if self.device == "cuda":
            torch.cuda.synchronize()

    def max_over_ranks(self, v: float) -> float:
        if self.ws == 1:
            return v
        import torch
        import torch.distributed as dist
        t = torch.tensor([v], device=self.device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_rank: float, steps: int, max_ms: float) -> float:
        """Whole-job throughput: the units every rank processed over the
        slowest rank's time."""
        return units_per_rank * self.ws * steps / (max_ms / 1e3)


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
    ranks = Ranks("nccl", "cuda")
    barrier, max_over_ranks = ranks.barrier, ranks.max_over_ranks

    n, D = args.n or N_ITEMS, args.dim or DIM
    P = n * (n - 1) // 2
    stream = torch.cuda.current_stream()
    pipes = measure_pipes()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    X = synth.vectors_grouped(n, D, seed=0, device="cuda")
    items = ap.Items.from_vectors(X, precisions=(ap.AP_PREC_SPLIT_BF16,))
    if args.k_split >= 0 or args.mma_ctas:
        items.set_plan(128, 256, 0, args.k_split, args.mma_ctas)
    plan = items.plan()
    k_split, mma_ctas = plan["k_split"], plan["mma_ctas"]
    gram_kernel = "gram_tc2_kernel" if mma_ctas == 2 else "gram_tc_kernel"
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
    value = ranks.job_rate(P, args.steps, ms)
    if items.last_device_error() != 0:
        raise RuntimeError("device wait timed out during the benchmark")

    pk, pk_kind = peaks()
    peak_tf = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    flops_launch = 3 * 2.0 * D * P          # three BF16 products per pair, 2 flops per MAC
    achieved_tf = flops_launch / (gram_avg / 1e3) / 1e12
    # the capture covers the default 8192 x 2^20 schedule only
    traffic = (GRAM_TRAFFIC_BYTES.get(gram_kernel)
               if (n, D, k_split) == (N_ITEMS, DIM, 64) else None)
    roofline = {"bound": "tensor", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved_tf / peak_tf, "traffic": traffic,
                "kernel": gram_kernel, "peak_kind": f"{pk_kind} bf16 sustained",
                "algorithmic_flops_per_launch": flops_launch}

    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3/fp32-acc/fp64-norm", "data": "synthetic",
            "config": {"workload": f"pearson_n{n}_d{D}", "n_items": n, "dim": D,
                       "pairs": P, "precision": "split-bf16", "k_split": k_split,
                       "mma_ctas": mma_ctas,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs (32 GiB raw + 32 GiB hi/lo) far larger than L2"},
            "roofline": roofline, "gram_ms": gram_avg,
            # per step: vec_shift, vec_split, slice_stats, vec_split over the rows
            # centred again (normally none), slice_stats, gram_tc, and the pass
            # that scales (split-K) or corrects (whole tiles) the pairs
            "gpu_launches": 7 * args.steps}
    if clk:
        line["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}

    # ---- FP32 CUDA-core comparator (same launch shape, Gram + epilogue) ----
    if not args.no_fp32:
        items32 = ap.Items.from_vectors(X, precisions=(ap.AP_PREC_FP32,))
        out32 = torch.empty(P, dtype=torch.float64, device="cuda")
        items32.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32, out=out32)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        clk32 = ClockSampler(local)
        clk32.start()
        e0.record(stream)
        items32.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_FP32, out=out32)
        e1.record(stream)
        torch.cuda.synchronize()
        c32 = clk32.stop()
        items32.close()
        f32_ms = e0.elapsed_time(e1)
        line["fp32_gram_ms"] = f32_ms
        line["split_vs_fp32_speedup"] = f32_ms / gram_avg
        # the comparator against its own roof: the FP32 FMA pipe (two flops
        # per FMA), at the FMA rate measured here and the clock it ran at
        mhz32 = c32["sm_mhz"] if c32 else pipes["ffma"]["sm_mhz"]
        peak32 = 2 * pipes["ffma"]["per_clk_per_sm"] * n_sm * mhz32 * 1e6 / 1e12
        ach32 = 2.0 * D * P / (f32_ms / 1e3) / 1e12
        line["fp32_roofline"] = {"bound": "alu", "achieved": ach32, "peak": peak32,
                                 "unit": "TFLOP/s", "frac": ach32 / peak32,
                                 "kernel": "gram_f32_kernel",
                                 "peak_kind": f"FP32 FMA {pipes['ffma']['per_clk_per_sm']:.1f}"
                                              "/clk/SM (ap_pipe_rate, this run) x 2 flops x "
                                              f"{n_sm} SMs x {mhz32:.0f} MHz (median during the "
                                              "comparator)",
                                 "algorithmic_flops": 2.0 * D * P}
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
        X = None
        torch.cuda.empty_cache()
        Xh = synth.vectors_grouped(n, D, seed=0, device="cuda").cpu().pin_memory()
        res_h = torch.empty(P, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ksteps = max(1, min(args.steps, 3))
        # the two calls in sequence: copy + pre-process, then the Gram
        items.update(Xh)
        items.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_SPLIT_BF16, out=out)
        res_h.copy_(out, non_blocking=True)
        barrier()
        e0.record(stream)
        for _ in range(ksteps):
            items.update(Xh)
            items.run_pairs(ap.AP_FN_PEARSON, ap.AP_PREC_SPLIT_BF16, out=out)
            res_h.copy_(out, non_blocking=True)
        e1.record(stream)
        barrier()
        seq_ms = max_over_ranks(e0.elapsed_time(e1))
        # the fused call: transfers overlapped with the Gram macro by macro
        items.load_and_run(Xh, out=out)
        res_h.copy_(out, non_blocking=True)
        barrier()
        e0.record(stream)
        for _ in range(ksteps):
            items.load_and_run(Xh, out=out)
            res_h.copy_(out, non_blocking=True)
        e1.record(stream)
        barrier()
        e_ms = max_over_ranks(e0.elapsed_time(e1))
        line["e2e_update_then_run_ms_per_step"] = seq_ms / ksteps
        line["e2e"] = {"value": P * ws * ksteps / (e_ms / 1e3), "unit": "pairs/s",
                       "h2d_bytes_per_step": int(n * D * 4),
                       "d2h_bytes_per_step": int(P * 8), "steps": ksteps,
                       "ms_per_step": e_ms / ksteps}
        # one more call with the task trace on (after the timed ones)
        items.set_trace(True)
        items.load_and_run(Xh, out=out)
        line["e2e"]["timeline"] = timeline_summary(items.trace())
        items.set_trace(False)
        Xh = res_h = None
    items.close()
    line["pipe_rates_per_clk_per_sm"] = {k: v["per_clk_per_sm"] for k, v in pipes.items()}
    if ws == 1 and not args.no_extra and (args.n, args.dim) == (0, 0):
        X = items = out = out32 = None
        torch.cuda.empty_cache()
        line["configs"] = extra_configs(args, pipes)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# SFU (MUFU) throughput of a GB300 SM, measured with independent chains of
# each instruction: ex2.approx 30.2 and rcp.approx 15.2 results per clock;
# the overlap kernels' roofline is 152 SMs x the SM clock seen during the run
# x the point-pair rate these allow (one rcp and one ex2 per point pair)
EX2_PER_CLK_PER_SM = 32
RCP_PER_CLK_PER_SM = 16
OOC_N, OOC_DIM, OOC_CACHE = 8192, 3 << 20, 48 << 30


def ooc_record(steps=3, warmup=1, policy=2, no_cpu=False, n=0, D=0, cache=0):
    """Out-of-core correlation: 8192 vectors of 3*2^20 FP32 (96 GiB) in pinned
    host memory streamed through a 48 GiB HBM slot cache (the host's 199 GB of
    RAM cannot hold the 16,384-vector, 192 GiB set pinned; set and cache are
    both halved, keeping their ratio).  Returns the JSON record."""
    import numpy as np
    import torch
    import synth
    import paper_2009_04755_gb300 as ap
    t_wall = time.perf_counter()
    n, D, cache = n or OOC_N, D or OOC_DIM, cache or OOC_CACHE
    P = n * (n - 1) // 2
    torch.cuda.set_device(0)
    Xh = torch.empty(n, D, dtype=torch.float32, pin_memory=True)
    chunk = 1024
    for r0 in range(0, n, chunk):
        rows = min(chunk, n - r0)
        Xd = synth.vectors_grouped(rows, D, seed=1000 + r0 // chunk, device="cuda")
        Xh[r0:r0 + rows].copy_(Xd)
        del Xd
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # the host link as measured here: macro-sized (3 GiB) pinned -> device
    # copies from eight places of the host set, best of them
    macro = 256 * D
    probe = torch.empty(macro, dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flat = Xh.view(-1)
    rates = []
    for k in range(9):
        off = (k * (n // 8) % (n - 256)) * D
        e0.record()
        probe.copy_(flat[off:off + macro], non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        if k:
            rates.append(macro * 4 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    link_gbs = max(rates)
    # the whole host set copied once, macro by macro, with nothing else
    # running: the link rate this buffer allows on average (its pages do not
    # all copy at the same rate)
    ring = [probe, torch.empty(macro, dtype=torch.float32, device="cuda")]
    cs = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(cs):
        e0.record(cs)
        for m in range(n // 256):
            ring[m % 2].copy_(flat[m * macro:(m + 1) * macro], non_blocking=True)
        e1.record(cs)
    torch.cuda.synchronize()
    whole_gbs = n * D * 4 / (e0.elapsed_time(e1) / 1e3) / 1e9
    del probe, ring
    items = ap.Items.from_vectors(Xh, slot_cache_bytes=cache)
    if policy:
        items.set_out_of_core_policy(policy)
    out = torch.empty(P, dtype=torch.float64, device="cuda")
    for _ in range(max(1, warmup)):
        items.run_pairs(out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0.record()
    for _ in range(steps):
        items.run_pairs(out=out)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    st = items.stats()
    h2d_gbs = st["h2d_bytes"] / (ms / 1e3) / 1e9
    # one more run with the task trace on (after the timed ones)
    items.set_trace(True)
    items.run_pairs(out=out)
    timeline = timeline_summary(items.trace())
    items.set_trace(False)
    line = {"metric": METRIC, "value": P / (ms / 1e3), "unit": "pairs/s", "n_gpus": 1,
            "steps": steps, "warmup": max(1, warmup), "ms_per_step": ms, "timeline": timeline,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3/fp32-acc/fp64-norm", "data": "synthetic",
            "config": {"workload": f"pearson_ooc_n{n}_d{D}", "n_items": n, "dim": D,
                       "host_bytes": n * D * 4, "slot_cache_bytes": cache,
                       "policy": ["resident+streamed", "recursive+lru",
                                  "column-slices"][policy]},
            "reuse_R": st["reuse_R"], "slot_hit_rate": st["slot_hit_rate"],
            "h2d_bytes_per_step": st["h2d_bytes"], "h2d_gbs": h2d_gbs,
            "roofline": {"bound": "link", "achieved": h2d_gbs, "peak": whole_gbs,
                         "unit": "GB/s", "frac": h2d_gbs / whole_gbs, "traffic": None,
                         "peak_kind": "the whole pinned host set copied once to the device, "
                                      "macro by macro, nothing else running (this run)"},
            "link_probe_gbs": {"min": min(rates), "median": statistics.median(rates),
                               "max": max(rates), "whole_set": whole_gbs},
            "frac_of_best_macro_copy": h2d_gbs / link_gbs,
            "compulsory_link_frac": (n * D * 4) / (ms / 1e3) / 1e9 / whole_gbs}
    if clk:
        line["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    if not no_cpu:
        # the oracle on every pair of a seeded sample of rows, read from the
        # pinned host set itself
        import oracle
        oracle.build()
        k = 24
        rows = sample_rows(n, k, seed=99)
        sub = Xh[torch.from_numpy(rows)].numpy()
        cores = os.cpu_count() or 1
        pi, pj, r_ref, secs = run_oracle_sample(sub, cores)
        gi, gj = rows[pi], rows[pj]
        p = torch.from_numpy(gi * n - gi * (gi + 1) // 2 + (gj - gi - 1)).cuda()
        line["max_abs_err_sampled"] = float(np.abs(out[p].cpu().numpy() - r_ref).max())
        line["cpu_baseline"] = {"value": len(pi) / secs, "unit": "pairs/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"all {len(pi)} pairs of {k} sampled vectors"}
    items.close()
    del Xh
    line["wall_s"] = time.perf_counter() - t_wall
    return line


def host_ram_bytes():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        return 0


def run_ooc_workload(args):
    print(json.dumps(ooc_record(args.steps, args.warmup, args.ooc_policy, args.no_cpu,
                                args.n, args.dim, int(args.ooc_cache_gib * (1 << 30)))),
          flush=True)
    return 0


def extra_configs(args, pipes):
    """The workloads besides the headline, each a bounded run inside the
    default benchmark so that one run carries all of them: the 2-D overlap of
    256 clouds (every pair checked against the oracle), 20 fused ascent steps
    on 1024 template clouds (teacher-forced check), the 3-D overlap of 20,000
    lognormal clouds (sampled check) and the out-of-core correlation (sampled
    check; skipped when the host cannot pin its 96 GiB)."""
    import torch
    out = {}
    plans = (("overlap2d_n256", 2000, 200, dict(full_oracle=True)),
             ("register2d_n1024", 5, 3, {}),
             ("overlap3d_n20000", 2, 1, {}))
    for wl, steps, warmup, kw in plans:
        try:
            out[wl] = cloud_record(wl, "overlap", steps, warmup, args.ref_pairs, "",
                                   args.no_cpu, pipes, **kw)
        except Exception as e:                    # reported, never hidden
            out[wl] = {"error": repr(e)}
        torch.cuda.empty_cache()
    need = OOC_N * OOC_DIM * 4 + (40 << 30)
    if host_ram_bytes() < need:
        out["pearson_ooc_n8192_d3145728"] = {
            "skipped": f"host RAM {host_ram_bytes() / 2**30:.0f} GiB < {need / 2**30:.0f} GiB "
                       "needed to pin the 96 GiB set"}
    else:
        try:
            out["pearson_ooc_n8192_d3145728"] = ooc_record(3, 1, 2, args.no_cpu)
        except Exception as e:
            out["pearson_ooc_n8192_d3145728"] = {"error": repr(e)}
    return out


def run_pearson_list_workload(args):
    """Pearson of a chosen list of pairs: 20,000 random pairs (either
    orientation) of the resident 8192 x 2^20 set.  Each call copies the
    touched row blocks of the split-BF16 arrays into row-major rows
    (list_rows_kernel), then runs one warp per pair over them
    (pearson_rows_kernel); both run inside the timed call.  The roofline is
    HBM bytes: both rows' hi and lo per pair, over the whole call's time."""
    import numpy as np
    import torch
    import synth
    import paper_2009_04755_gb300 as ap
    torch.cuda.set_device(0)
    n, D = args.n or N_ITEMS, args.dim or DIM
    L = 20000
    X = synth.vectors_grouped(n, D, seed=0, device="cuda")
    items = ap.Items.from_vectors(X, precisions=(ap.AP_PREC_SPLIT_BF16,))
    rng = np.random.default_rng(11)
    pi = rng.integers(0, n, L).astype(np.int32)
    pj = ((pi + rng.integers(1, n, L)) % n).astype(np.int32)
    out = torch.empty(L, dtype=torch.float64, device="cuda")
    for _ in range(max(args.warmup, 3)):
        items.run_pairs_list(pi, pj, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        items.run_pairs_list(pi, pj, out=out)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    Dp = (D + 63) // 64 * 64
    bytes_step = L * 2 * Dp * 4                       # both rows' hi + lo per pair
    pk, pk_kind = peaks()
    peak = pk.get("hbm_gbs", 6800.0)
    gbs = bytes_step / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": L / (ms / 1e3), "unit": "pairs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3/fp32-acc/fp64-norm", "data": "synthetic",
            "config": {"workload": f"pearson_list_n{n}_d{D}", "n_items": n, "dim": D,
                       "listed_pairs": L, "precision": "split-bf16",
                       "l2": "each step reads 168 GB of rows, far larger than L2"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "traffic": None,
                         "kernel": "pearson_rows_kernel (with list_rows_kernel's row-major "
                                   "copy and the host sort, over the whole call)",
                         "peak_kind": f"{pk_kind} HBM copy",
                         "algorithmic_bytes_per_step": bytes_step},
            "gpu_launches": 2 * args.steps}
    if clk:
        line["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    if not args.no_cpu:
        import oracle
        k = 200
        rows = np.unique(np.concatenate([pi[:k], pj[:k]]))
        sub = X[torch.from_numpy(rows).cuda()].cpu().numpy()
        remap = {r: q for q, r in enumerate(rows)}
        cores = os.cpu_count() or 1
        oracle.build()
        t0 = time.perf_counter()
        ref = oracle.pearson(sub, [remap[a] for a in pi[:k]], [remap[b] for b in pj[:k]],
                             n_threads=cores)
        secs = time.perf_counter() - t0
        line["max_abs_err_sampled"] = float(np.abs(out[:k].cpu().numpy() - ref).max())
        line["cpu_baseline"] = {"value": k / secs, "unit": "pairs/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"the first {k} listed pairs (their rows' statistics "
                                          "included)"}
    items.close()
    print(json.dumps(line), flush=True)
    return 0


SPARSE_N, SPARSE_DIM = 2500, 20 ** 6
# shared-memory / L1 data path of an SM: 128 bytes per clock; a probe of the
# sparse cosine moves 12 (a 4-byte gather from the dense chunk + the 8-byte
# entry it multiplies)
L1_BYTES_PER_CLK_PER_SM = 128
SPARSE_BYTES_PER_PROBE = 12


def run_sparse_workload(args):
    """Cosine of sparse composition vectors: 2500 items (Table I's
    bioinformatics set) over 20^6 k-mer codes, 1e5-1.8e6 entries each."""
    import numpy as np
    import torch
    import synth
    import paper_2009_04755_gb300 as ap
    torch.cuda.set_device(0)
    n = args.n or SPARSE_N
    off, idx, val = synth.sparse_cv(n, dim=SPARSE_DIM, seed=0, device="cuda", as_torch=True)
    nnz = np.diff(off).astype(np.float64)
    P = n * (n - 1) // 2
    # the kernel streams row j's entries for every pair (i < j)
    probes = float((nnz * np.arange(n)).sum())
    items = ap.Items.from_sparse(off, idx, val, SPARSE_DIM)
    out = torch.empty(P, dtype=torch.float64, device="cuda")
    for _ in range(max(args.warmup, 3)):
        items.run_pairs(ap.AP_FN_COSINE, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        items.run_pairs(ap.AP_FN_COSINE, out=out)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    sm_mhz = clk["sm_mhz"] if clk else 2070.0
    achieved = probes * SPARSE_BYTES_PER_PROBE / (ms / 1e3) / 1e9
    peak = L1_BYTES_PER_CLK_PER_SM * 152 * sm_mhz * 1e6 / 1e9
    line = {"metric": METRIC, "value": P / (ms / 1e3), "unit": "pairs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-products/fp64-sums", "data": "synthetic",
            "config": {"workload": f"cosine_sparse_n{n}", "n_items": n, "dim": SPARSE_DIM,
                       "nnz_total": int(nnz.sum()), "pairs": P, "probes": probes},
            "probes_per_s": probes / (ms / 1e3),
            "roofline": {"bound": "l1", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "sparse_cos_kernel",
                         "peak_kind": "128 B/clk/SM shared/L1 data path x 152 SMs x median SM "
                                      "clock; 12 B per probe"},
            "gpu_launches": args.steps}
    if clk:
        line["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    if not args.no_cpu:
        import oracle
        rng = np.random.default_rng(7)
        k = 200
        rows = np.sort(rng.choice(n, size=2 * k, replace=False))
        pi, pj = rows[0::2], rows[1::2]
        # the sampled rows to the host, renumbered
        sub = np.unique(np.concatenate([pi, pj]))
        loc = {r: q for q, r in enumerate(sub)}
        soff = np.zeros(len(sub) + 1, np.int64)
        np.cumsum(nnz[sub].astype(np.int64), out=soff[1:])
        sidx = torch.cat([idx[off[r]:off[r + 1]] for r in sub]).cpu().numpy()
        sval = torch.cat([val[off[r]:off[r + 1]] for r in sub]).cpu().numpy()
        li = np.array([loc[r] for r in pi]); lj = np.array([loc[r] for r in pj])
        cores = os.cpu_count() or 1
        oracle.build()
        t0 = time.perf_counter()
        ref = oracle.sparse_cosine(soff, sidx, sval, li, lj, n_threads=cores)
        secs = time.perf_counter() - t0
        p = torch.from_numpy(pi * n - pi * (pi + 1) // 2 + (pj - pi - 1)).cuda()
        got = out[p].cpu().numpy()
        line["max_abs_err_sampled"] = float(np.abs(got - ref).max())
        line["cpu_baseline"] = {"value": len(pi) / secs, "unit": "pairs/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"{len(pi)} random pairs of the workload"}
    items.close()
    print(json.dumps(line), flush=True)
    return 0


ENC_N, ENC_DIM = 2048, 1 << 20


def run_encoded_workload(args):
    """The load pipeline with its parse stage: 2048 rows of 2^20 FP32 given
    encoded (XOR + varint, ~4.5 bytes a value), decoded on the host's cores
    into a 4 GiB pinned host cache (the second-level cache) and streamed
    through a 3 GiB HBM slot cache (three 256-row macros of the eight), so
    the device cache reloads macros and the host cache serves part of them."""
    import numpy as np
    import torch
    import synth
    import paper_2009_04755_gb300 as ap
    torch.cuda.set_device(0)
    n, D = args.n or ENC_N, ENC_DIM
    P = n * (n - 1) // 2
    X = synth.vectors_grouped(n, D, seed=0, device="cuda").cpu().numpy()
    t0 = time.perf_counter()
    blobs = [ap.binding.encode_vector(X[i]) for i in range(n)]
    enc_s = time.perf_counter() - t0
    enc_bytes = sum(len(b) for b in blobs)
    slot = 256 * D * 4
    items = ap.Items.from_encoded(blobs, D, slot_cache_bytes=3 * slot,
                                  host_cache_bytes=4 * slot)
    out = torch.empty(P, dtype=torch.float64, device="cuda")
    for _ in range(max(args.warmup, 3)):
        items.run_pairs(out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    parsed, hits = 0, []
    for _ in range(args.steps):
        items.run_pairs(out=out)
        st = items.stats()
        parsed += st["parsed_rows"]
        hits.append(st["host_hit_rate"])
    e1.record()
    torch.cuda.synchronize()
    wall_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    cores = os.cpu_count() or 1
    # the parse stage's own rate: one core decoding rows, times the cores
    sample = blobs[:8]
    t1 = time.perf_counter()
    for b in sample:
        ap.binding.decode_vector(b, D)
    one_core = len(sample) * D * 4 / (time.perf_counter() - t1) / 1e9
    parse_gbs = parsed / args.steps * D * 4 / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": P / (ms / 1e3), "unit": "pairs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3/fp32-acc/fp64-norm", "data": "synthetic",
            "config": {"workload": f"pearson_encoded_n{n}_d{D}", "n_items": n, "dim": D,
                       "encoded_bytes": enc_bytes, "slot_cache_bytes": 3 * slot,
                       "host_cache_bytes": 4 * slot, "codec": "xor-varint",
                       "parse_threads": cores},
            "parsed_rows_per_step": parsed / args.steps,
            "host_hit_rate": float(np.mean(hits)) if hits else 0.0,
            "item_loads_per_step": st["item_loads"], "reuse_R": st["reuse_R"],
            "parse_gbs": parse_gbs, "wall_ms_per_step": wall_ms,
            "roofline": {"bound": "host parse", "achieved": parse_gbs,
                         "peak": one_core * cores, "unit": "GB/s",
                         "frac": parse_gbs / (one_core * cores), "traffic": None,
                         "peak_kind": "one core's decode rate of a row (measured here) "
                                      "x the host's cores"},
            "encode_s": enc_s, "gpu_launches": None}
    if clk:
        line["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    items.close()
    print(json.dumps(line), flush=True)
    return 0


def timeline_summary(tr):
    """Busy time per stream, the link rate while copying and how much of the
    copying overlapped the Gram, from one traced run's tasks (ap_get_trace)."""
    def union(iv):
        tot, cur = 0.0, None
        for a, b in sorted(iv):
            if cur is None or a > cur[1]:
                if cur:
                    tot += cur[1] - cur[0]
                cur = [a, b]
            else:
                cur[1] = max(cur[1], b)
        return tot + (cur[1] - cur[0] if cur else 0.0)

    def ivs(stage):
        return [(e["start_ms"], e["end_ms"]) for e in tr if e["stage"] == stage]

    if not tr:
        return None
    total = max(e["end_ms"] for e in tr)
    cp, gr, pp = ivs("copy"), ivs("gram"), ivs("preprocess")
    both = union([(max(a, c), min(b, d)) for a, b in cp for c, d in gr if min(b, d) > max(a, c)])
    copy_ms = union(cp)
    nbytes = sum(e["bytes"] for e in tr)
    return {"total_ms": total, "tasks": len(tr),
            "copy_busy_ms": copy_ms, "preprocess_busy_ms": union(pp), "gram_busy_ms": union(gr),
            "copy_overlapped_by_gram_ms": both,
            "h2d_gbs_while_copying": nbytes / (copy_ms / 1e3) / 1e9 if copy_ms else None,
            "first_gram_start_ms": min(a for a, _ in gr) if gr else None,
            "after_last_copy_ms": total - max(b for _, b in cp) if cp else None}


def measure_pipes():
    """Issue rates of the FP32 FMA pipe and the MUFU ex2 / rcp instructions
    on this GPU, measured here by the library's probe (ap_pipe_rate): results
    per clock per SM, the denominators of the CUDA-core kernels' rooflines."""
    import paper_2009_04755_gb300 as ap
    out = {}
    for name, k in (("ffma", ap.binding.PIPE_FMA), ("ex2", ap.binding.PIPE_EX2),
                    ("rcp", ap.binding.PIPE_RCP), ("ffma2", ap.binding.PIPE_FMA2)):
        r = ap.binding.pipe_rate(k)
        out[name] = {"per_clk_per_sm": r["per_clk_per_sm"], "sm_mhz": r["sm_mhz"]}
    return out


def mufu_roof(pipes, sm_mhz, n_sm):
    """The overlap kernels' bound: one rcp and one ex2 per point pair on the
    SM's MUFU pipe.  Returns (peak MUFU results/s in units of 1e12, point
    pairs per clock per SM, how the rates were obtained)."""
    if pipes:
        rcp, ex2 = pipes["rcp"]["per_clk_per_sm"], pipes["ex2"]["per_clk_per_sm"]
        kind = "ap_pipe_rate measured in this run"
    else:
        rcp, ex2 = RCP_PER_CLK_PER_SM, EX2_PER_CLK_PER_SM
        kind = "rates of an earlier probe"
    pp = 1.0 / (1.0 / rcp + 1.0 / ex2)
    return 2.0 * pp * n_sm * sm_mhz * 1e6 / 1e12, pp, \
        f"one rcp ({rcp:.1f}/clk/SM) + one ex2 ({ex2:.1f}/clk/SM) per point pair ({kind}): " \
        f"{2 * pp:.1f} MUFU results/clk/SM x {n_sm} SMs x median SM clock"


def cloud_record(wl, fn_name="overlap", steps=5, warmup=3, ref_pairs=2000, plan="",
                 no_cpu=False, pipes=None, n_override=0, full_oracle=False):
    """Point-cloud workloads: overlap cost (2-D n=256, 3-D lognormal n=20000),
    batched registration (2-D n=1024, 20 fused ascent steps per step), the
    particle scores; returns the JSON record.  full_oracle: every pair is
    checked against the oracle (the 256-cloud workload), else a seeded sample;
    registration is checked teacher-forced (f and its gradient at the GPU's
    own parameters after the 20 steps)."""
    import numpy as np
    import torch
    import synth
    import paper_2009_04755_gb300 as ap

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    t_wall = time.perf_counter()
    if wl == "overlap2d_n256":
        c = synth.clouds_uniform(n=256, dim=2, size=(64, 128), seed=0)
    elif wl == "particles2d_n256":
        # the paper's microscopy set: 256 particles of 1000-2000 localisations
        c = synth.clouds_uniform(n=256, dim=2, size=(1000, 2000), sigma=(0.01, 0.03), seed=0)
    elif wl == "register_particles2d_n256":
        # all-to-all registration of 256 particles of 1000-2000 localisations
        # (8 templates of 2000 points, random poses): 20 ascent steps on the
        # overlap, then the GMM L2 distance at the registered poses
        c = synth.clouds_templates(n=256, template_pts=2000, size=(1000, 2000),
                                   sigma=(0.01, 0.03), seed=0)
    elif wl == "overlap3d_n20000":
        c = synth.clouds_lognormal(n=n_override or 20000, dim=3, seed=0)
    else:   # register2d_n1024 and its pair-list form
        c = synth.clouds_templates(n=1024, seed=0)
    n = len(c["offsets"]) - 1
    P = n * (n - 1) // 2
    sizes = np.diff(c["offsets"]).astype(np.float64)
    point_pairs = (sizes.sum() ** 2 - (sizes ** 2).sum()) / 2
    listed = wl == "register2d_n1024_list"
    if listed:
        # a seeded quarter of the pairs, in random order and either orientation
        rng = np.random.default_rng(7)
        li, lj = np.triu_indices(n, 1)
        keep = rng.permutation(P)[:P // 4]
        flip = rng.random(len(keep)) < 0.5
        lpi = np.where(flip, lj[keep], li[keep]).astype(np.int32)
        lpj = np.where(flip, li[keep], lj[keep]).astype(np.int32)
        P = len(keep)
        point_pairs = float((sizes[lpi] * sizes[lpj]).sum())
    items = ap.Items.from_clouds(c)
    reg = wl in ("register2d_n1024", "register_particles2d_n256", "register2d_n1024_list")
    if plan:
        bi, bp, rr = (int(v) for v in plan.split(","))
        items.set_plan(bi, bp, rr)
        tuned = items.plan()
    else:
        tuned = items.tune(1 if reg else 0)
    stream = torch.cuda.current_stream()
    out = torch.empty(P, dtype=torch.float32, device="cuda")
    n_asc = 20
    prm = torch.zeros(P, 3, device="cuda")

    fn = {"overlap": ap.AP_FN_OVERLAP, "gmm_l2": ap.AP_FN_GMM_L2,
          "bhattacharyya": ap.AP_FN_BHATTACHARYYA}[fn_name]

    def step():
        if listed:
            prm.zero_()
            items.ascent_list(lpi, lpj, prm, n_asc, 1e-3)
        elif reg:
            prm.zero_()
            items.ascent(prm, n_asc, 1e-3)
            if wl == "register_particles2d_n256":
                items.run_pairs(ap.AP_FN_GMM_L2, params=prm, out=out)
        else:
            items.run_pairs(fn, out=out)

    for _ in range(max(warmup, 1)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    evals = n_asc + (wl == "register_particles2d_n256") if reg else 1   # pair evaluations per step
    units = P * (n_asc if wl in ("register2d_n1024", "register2d_n1024_list") else 1)
    mufu = 2.0 * point_pairs * evals
    sm_mhz = clk["sm_mhz"] if clk else 2070.0
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peak, _, peak_kind = mufu_roof(pipes, sm_mhz, n_sm)
    achieved = mufu / (ms / 1e3) / 1e12
    line = {"metric": METRIC, "value": units / (ms / 1e3),
            "unit": {"register2d_n1024": "pair-steps/s", "register2d_n1024_list": "pair-steps/s",
                     "register_particles2d_n256": "pair registrations/s"}.get(wl, "pairs/s"),
            "n_gpus": 1, "steps": steps, "warmup": max(warmup, 1), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"overlap3d_n{n}" if wl == "overlap3d_n20000" else wl,
                       "n_items": n, "pairs": P, "point_pairs": point_pairs,
                       "pair_function": {"register2d_n1024": "ascent (20 steps)",
                                         "register2d_n1024_list":
                                             "ascent (20 steps) on a listed quarter of the pairs",
                                         "register_particles2d_n256":
                                             "ascent (20 steps) + gmm_l2"}.get(wl, fn_name),
                       "plan": tuned},
            "point_pairs_per_s": point_pairs * evals / (ms / 1e3),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TMUFU/s", "frac": achieved / peak, "traffic": None,
                         "kernel": "overlap_kernel", "peak_kind": peak_kind},
            "gpu_launches": steps * evals}
    if clk:
        line["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    if not no_cpu:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        rng = np.random.default_rng(7)
        if full_oracle:
            pi, pj = oracle.all_pairs(n)
        else:
            k = ref_pairs
            pi = rng.integers(0, n - 1, 4 * k)
            pj = rng.integers(0, n, 4 * k)
            keep = pi < pj
            pi, pj = pi[keep][:k], pj[keep][:k]
        if listed:                             # a sample of the listed pairs, as listed
            sel = rng.permutation(P)[:ref_pairs]
            pi, pj = lpi[sel], lpj[sel]
        pidx = None if listed else torch.from_numpy(pi * n - pi * (pi + 1) // 2 + (pj - pi - 1)).cuda()
        t0 = time.perf_counter()
        if reg and not listed:
            # teacher-forced: the oracle's f and gradient at the GPU's own
            # parameters after the 20 ascent steps (one evaluation, timed)
            prm_s = prm[pidx].double().cpu().numpy()
            f_ref, g_ref = oracle.overlap_grad(c, pi, pj, prm_s, n_threads=cores)
        elif listed:
            f_ref, g_ref = oracle.overlap_grad(c, pi, pj, None, n_threads=cores)
        elif fn_name == "gmm_l2":
            f_ref = oracle.gmm_l2(c, pi, pj, n_threads=cores)
        elif fn_name == "bhattacharyya":
            f_ref = oracle.bhattacharyya(c, pi, pj, n_threads=cores)
        else:
            f_ref, kappa, bound = oracle.overlap(c, pi, pj, n_threads=cores, with_cond=True)
        secs = time.perf_counter() - t0
        if wl == "register_particles2d_n256":
            secs *= evals                      # the sample's time for a whole registration
            f_ref = oracle.gmm_l2(c, pi, pj, params=prm_s, n_threads=cores)
            items.run_pairs(ap.AP_FN_GMM_L2, params=prm, out=out)
            got = out[pidx].double().cpu().numpy()
        elif reg and not listed:
            f_gpu = items.run_pairs(ap.AP_FN_OVERLAP, params=prm)
            g_gpu, _ = items.backward(params=prm)
            got = f_gpu[pidx].double().cpu().numpy()
            gg = g_gpu[pidx].double().cpu().numpy()
            scale = np.maximum(np.abs(g_ref).max(1), 1e-6 * sizes[pi] * sizes[pj])
            line["max_grad_err_normwise_sampled"] = float(
                (np.abs(gg - g_ref).max(1) / scale).max())
        elif listed:
            got = items.run_pairs_list(pi, pj).double().cpu().numpy()
        else:
            got = out[pidx].double().cpu().numpy()
        rel = np.abs(got - f_ref) / np.abs(f_ref)
        if not reg and fn_name == "overlap":
            # conditioning-aware: 1e-5 relative where the FP32 evaluation is
            # well conditioned, the oracle's FP32 error scale elsewhere
            good = (kappa * 2.0 ** -23 * 8 <= 1e-5) & (f_ref >= 1e-30)
            line["max_rel_err_sampled"] = float(rel[good].max(initial=0.0))
            line["pairs_checked"] = int(len(pi))
            line["pairs_beyond_tolerance"] = int(
                (rel[good] > 1e-5).sum() + (np.abs(got - f_ref)[~good] >
                                           np.maximum(3 * bound[~good], 1e-5 * f_ref[~good])).sum())
        else:
            line["max_rel_err_sampled"] = float(rel.max())
        unit = line["unit"]
        if wl in ("register2d_n1024", "register2d_n1024_list"):
            cpu_v, smp = len(pi) * n_asc / (secs * n_asc), "one ascent evaluation of"
        elif wl == "register_particles2d_n256":
            cpu_v, smp = len(pi) / secs, f"one ascent evaluation (x{evals}) of"
        else:
            cpu_v, smp = len(pi) / secs, "all of"
        line["cpu_baseline"] = {"value": cpu_v, "unit": unit, "cores": cores, "kind": "oracle",
                                "sample": f"{smp} {len(pi)} "
                                          f"{'' if full_oracle else 'random '}pairs of the workload"}
    items.close()
    line["wall_s"] = time.perf_counter() - t_wall
    return line


def run_cloud_workload(args):
    wl = args.workload
    steps = args.steps
    line = cloud_record(wl, args.fn, steps, args.warmup, args.ref_pairs, args.plan, args.no_cpu,
                        measure_pipes(), args.n, full_oracle=(wl == "overlap2d_n256"))
    print(json.dumps(line), flush=True)
    return 0


# workloads whose step is far shorter than the 200 ms clock sampling period
SHORT_STEP_WORKLOADS = {"overlap2d_n256": 5000}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--workload", default="pearson_n8192_d1048576",
                    choices=["pearson_n8192_d1048576", "overlap2d_n256", "overlap3d_n20000",
                             "register2d_n1024", "register2d_n1024_list",
                             "pearson_list_n8192_d1048576", "pearson_ooc_n8192_d3145728",
                             "particles2d_n256", "register_particles2d_n256",
                             "cosine_sparse_n2500", "pearson_encoded_n2048_d1048576"])
    ap.add_argument("--fn", default="overlap", choices=["overlap", "gmm_l2", "bhattacharyya"],
                    help="pair function of the cloud workloads")
    ap.add_argument("--ref-pairs", type=int, default=2000)
    ap.add_argument("--n", type=int, default=0,
                    help="item count override (smaller cases for profiling)")
    ap.add_argument("--dim", type=int, default=0, help="vector length override")
    ap.add_argument("--plan", default="",
                    help="cloud tile plan block_items,block_pts,reg_r instead of tuning")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 5; 5000 for the 0.2 ms overlap2d_n256 step, so "
                         "that the timed region lasts long enough to sample its clocks)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-rows", type=int, default=512,
                    help="vectors in the oracle's bounded sample (all their pairs)")
    ap.add_argument("--k-split", type=int, default=-1,
                    help="Pearson Gram schedule: column ranges per tile (0 whole tiles; "
                         "-1 the library default)")
    ap.add_argument("--mma-ctas", type=int, default=0, choices=[0, 1, 2],
                    help="Pearson Gram: CTAs per tensor-core MMA (1 one CTA per tile, 2 CTA "
                         "pairs; 0 the library default)")
    ap.add_argument("--ooc-policy", type=int, default=2, choices=[0, 1, 2],
                    help="out-of-core schedule: 0 resident+streamed, 1 recursive order + LRU, "
                         "2 column slices")
    ap.add_argument("--ooc-cache-gib", type=float, default=0.0,
                    help="out-of-core slot cache size override (GiB; with --n/--dim for "
                         "smaller cases)")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads' records in the default run")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = SHORT_STEP_WORKLOADS.get(args.workload, 5) if args.impl == "ours" else 5
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "pearson_ooc_n8192_d3145728":
        return run_ooc_workload(args)
    if args.workload == "cosine_sparse_n2500":
        return run_sparse_workload(args)
    if args.workload == "pearson_list_n8192_d1048576":
        return run_pearson_list_workload(args)
    if args.workload == "pearson_encoded_n2048_d1048576":
        return run_encoded_workload(args)
    if args.workload != "pearson_n8192_d1048576":
        return run_cloud_workload(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
