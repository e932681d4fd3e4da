"""Benchmark: CP-ALS over CSF on the 3-mode power-law tensor of NETFLIX shape.

Workload (default): 480,000 x 18,000 x 2,000, 1e8 distinct non-zeros, Zipf(1.1)
per mode through a random permutation, values lognormal(0,1), rank 16, FP32
factor gathers (FP32 accumulate, FP64 R x R solve). One step = one CP-ALS
iteration (Algorithm 1): per mode an MTTKRP over the CSF rooted at that mode,
the normal-equation solve, normalisation, then the fit, with the CSFs
resident in HBM (they are built once, as the paper's pre-processing).

value  = whole-job MTTKRP work rate, N_modes * nnz * R per iteration / time,
         in Gnnz*R/s (summed over ranks: each rank runs an independent replica).
e2e    = the same metric through the one-shot C-ABI call (sptt_cpd_als) from
         pinned host buffers: host->device copy of the COO, sort/CSF builds,
         the ALS iterations and the copy of the factors back, all timed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MTTKRP Gnnz·R/s, %HBM peak; CP-ALS s/iter mixed vs FP32 at Δfit≤1e-4"
UNIT = "Gnnz·R/s"
WORKLOAD = "powerlaw3 480000x18000x2000 nnz=1e8 zipf1.1+perm lognormal(0,1)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--rank", type=int, default=16)
    p.add_argument("--nnz", type=int, default=100_000_000)
    p.add_argument("--seed", type=int, default=2)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--e2e-iters", type=int, default=20)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--extras", default="precision,mixed4,mixed_vs_oracle,batched,sched,tiling",
                   help="comma list of the extra measurements to run (default: all): precision (FP32 vs BF16 "
                        "at R = 16, 32), mixed4 (4-mode R = 64 mixed vs FP32), mixed_vs_oracle, batched (512 "
                        "tensors, autotuned plan), sched (learned scheduler vs the default), tiling (R = 32)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--extra-one-csf", action="store_true",
                   help="also time one CSF for all modes (non-root MTTKRPs with privatised hot rows)")
    p.add_argument("--batch-count", type=int, default=512)
    p.add_argument("--sched-heldout", type=int, default=40)
    p.add_argument("--variant", type=int, default=0, help="MTTKRP kernel variant for every mode (0 = default)")
    p.add_argument("--chunk", type=int, default=0, help="MTTKRP chunk size (0 = default)")
    p.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                   help="factor gathers of the timed CP-ALS iterations (bf16: FP32 accumulation, FP64 solve)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist, device):
    """The maximum of a per-rank number over all ranks (x itself without a
    process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput in G units/s: every rank's units over the slowest
    rank's time (replicas: the per-rank work is fixed, so this is weak
    scaling)."""
    return units_per_rank * world / seconds / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample
# ---------------------------------------------------------------------------
def cpu_oracle_rate(t_cpu_inds, t_cpu_vals, dims, R, seconds, threads=1):
    """Times one oracle CP-ALS iteration on a prefix sample sized for about
    `seconds` of CPU work, on `threads` host threads (the oracle's threaded
    MTTKRP and row loops). Returns (Gnnz*R/s, seconds, sample size)."""
    import numpy as np

    import oracle
    oracle.set_threads(threads)
    nnz = t_cpu_vals.shape[0]

    def run(s):
        inds = [np.ascontiguousarray(x[:s]) for x in t_cpu_inds]
        vals = np.ascontiguousarray(t_cpu_vals[:s])
        t0 = time.perf_counter()
        oracle.cpd_als(inds, vals, dims, R, 1, seed=1, coalesce_first=False)
        return time.perf_counter() - t0

    # the iteration has a fixed part (Grams over all rows, the dense solve),
    # so the sample is rescaled until its time reaches the target
    s, t = min(nnz, 500_000), None
    t = run(s)
    for _ in range(3):
        if t >= 0.6 * seconds or s >= nnz:
            break
        s = int(min(nnz, s * seconds / max(t, 1e-3)))
        t = run(s)
    rate = len(dims) * s * R / t / 1e9
    return rate, t, s


def reference_arm(args, rank, world):
    """--impl reference: the FP64 oracle timed on the host cores, rank 0 only."""
    if rank != 0:
        return
    import numpy as np
    import torch

    import tensorgen
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = tensorgen.powerlaw3(seed=args.seed, device=dev, nnz=args.nnz)
    inds = [x.cpu().numpy() for x in t.inds]
    vals = t.vals.cpu().numpy()
    del t
    import oracle
    R = args.rank
    cores, model = host_cpu()
    threads = oracle.set_threads(cores)
    # one step = one oracle CP-ALS iteration on a bounded prefix sample
    budget = max(3.0, 150.0 / max(1, args.steps + args.warmup))
    _, t1, s = cpu_oracle_rate(inds, vals, [480_000, 18_000, 2_000], R, min(budget, 15.0), threads)
    sub_i = [np.ascontiguousarray(x[:s]) for x in inds]
    sub_v = np.ascontiguousarray(vals[:s])
    dims = [480_000, 18_000, 2_000]
    for _ in range(args.warmup):
        oracle.cpd_als(sub_i, sub_v, dims, R, 1, seed=1, coalesce_first=False)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.cpd_als(sub_i, sub_v, dims, R, 1, seed=1, coalesce_first=False)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = 3 * s * R * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "rank": R, "sample_nnz": s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "host_cores": cores, "cpu_model": model,
                         "sample": "one CP-ALS iteration (3 MTTKRPs + solve + fit) of the FP64 C oracle "
                                   "on the first %d non-zeros, %d threads" % (s, threads)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def byte_model(csf, dims, R, distinct, s_f=4):
    """Algorithmic bytes of one root-mode MTTKRP: values and leaf indices,
    fids/fptr of the upper levels, each distinct factor row once per level,
    and the output write."""
    n = csf.nmodes
    nnz = csf.nfibs[-1]
    b = nnz * (4 + 4)
    for l in range(n - 1):
        b += csf.nfibs[l] * (4 + 4)
    for l in range(1, n):
        b += distinct[csf.order[l]] * R * s_f
    b += dims[csf.root] * R * 4
    return b


def flop_model(csf, R):
    nnz = csf.nfibs[-1]
    return 2 * R * (nnz + sum(csf.nfibs[1:-1]))


def every_gather_model(csf, R, s_f=4):
    """Upper byte model: every factor-row gather from memory (no reuse)."""
    return sum(csf.nfibs[1:]) * R * s_f


# DRAM bytes (read + write) per launch of the default MTTKRP kernels, from
# one ncu capture at 3.4e7 non-zeros of this workload (roots 0, 1, 2; at this
# size the default rule picks the kernels it picks at 1e8: the table kernel
# for roots 0 and 1, the select walk for root 2); the traffic is dominated by
# the leaf-record stream, so it is scaled to other sizes by the number of
# non-zeros.
NCU_TRAFFIC = {"kernel": "mttkrp_table_kernel<3, float, 2, 1024, 16> (roots 0, 1), "
                         "mttkrp_select_kernel<3, float, 2, 2, 32> (root 2)",
               "nnz": 34_000_000, "bytes": [657.552896e6, 764.358144e6, 740.582912e6]}
# The same for the default BF16-gather kernels (the same rule: the BF16 table
# kernel at roots 0 and 1, variant 13 at root 2).
NCU_TRAFFIC_BF16 = {"kernel": "mttkrp_table_kernel<3, __nv_bfloat16, 4, 512, 16> (roots 0, 1), "
                              "mttkrp_select_kernel<3, __nv_bfloat16, 4, 2, 16> (root 2)",
                    "nnz": 34_000_000, "bytes": [648.869632e6, 664.093696e6, 639.894784e6]}


def input_checksum(t):
    """An order-independent integer fingerprint of a COO tensor (the same
    tensor gives the same value on any machine): per mode the sum of
    (index + 1) times a mode constant, plus the sum of the values' bit
    patterns, wrapped to 64 bits."""
    import torch
    h = 0
    for m, x in enumerate(t.inds):
        h += int(((x.long() + 1) * (2654435761 * (m + 1) + 1)).sum().item())
    h += int(t.vals.contiguous().view(torch.int32).long().sum().item())
    return "%016x" % (h % (1 << 64))


def fp32_peak_tflops(dev, sm_mhz=None):
    """FP32 FMA peak from the unit counts and the clock: the device's SM
    count x 128 FP32 lanes x 2 flops x the maximum SM clock (from
    MEASURED_PEAKS.json when present, else 2,070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if sm_mhz is None:
        sm_mhz = 2070.0
        path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(path):
            with open(path) as f:
                sm_mhz = float(json.load(f).get("sm_max_mhz", sm_mhz))
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12, sms, sm_mhz


def host_cpu():
    """(logical cores, CPU model) of this host: lscpu's vendor and model name,
    else /proc/cpuinfo's model name."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        kv = {}
        for line in out.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                kv.setdefault(k.strip().lower(), v.strip())
        parts = [kv.get("vendor id"), kv.get("model name")]
        model = " ".join(p for p in parts if p) or None
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.split(":")[0].strip().lower() == "model name":
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return os.cpu_count() or 1, model or "unknown"


def batched_extra(args, dev):
    """The batched workload: 512 tensors (3/4 modes, log-uniform sizes), R = 16,
    15 iterations, one persistent launch per run, replayed from a CUDA graph;
    against the same tensors decomposed one after another."""
    import torch

    import paper_1812_05961_gb300 as sptt
    import tensorgen
    R, iters = 16, 15
    specs = tensorgen.batch_tensor_specs(args.batch_count, seed=4)
    t0 = time.time()
    tensors = []
    for i, (dims, nnz) in enumerate(specs):
        x = tensorgen.batch_member(dims, nnz, seed=1000 + i, device=dev)
        tensors.append((x.dims, x.inds, x.vals))
    gen_s = time.time() - t0
    work = sum(len(d) * int(v.numel()) * R for d, _, v in tensors) * iters
    # byte model of one MTTKRP sweep over every tensor and mode (the batch's
    # CSFs take the ascending level order): values and leaf indices, fids and
    # fptr of the upper levels, each distinct factor row once, the output rows
    sweep_bytes = 0
    for d, inds, v in tensors:
        n = len(d)
        distinct = [int(torch.unique(x).numel()) for x in inds]
        for root in range(n):
            order = [root] + sorted((m for m in range(n) if m != root), key=lambda m: (d[m], m))
            key = torch.zeros_like(inds[0], dtype=torch.int64)
            fib = 0
            for l in range(n - 1):
                key = key * int(d[order[l]]) + inds[order[l]].long()
                fib += int(torch.unique(key).numel())
            sweep_bytes += int(v.numel()) * 8 + fib * 8 + sum(distinct[order[l]] for l in range(1, n)) * R * 4
            sweep_bytes += int(d[root]) * R * 4
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        t0 = time.time()
        b = sptt.Batch(tensors, R, seed=1, use_graph=1, plan=1)
        create_s = time.time() - t0
        sched, tuned_ms, ncand = b.schedule()
        b.init()
        b.run(iters)  # direct launch
        b.run(iters)  # captured
        grid, chunks, tiles = b.info()
        ph0 = sptt.sptt_batch_phase_ms(b.handle)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        ev0.record(side)
        for _ in range(reps):
            b.run(iters)
        ev1.record(side)
        torch.cuda.synchronize()
        batched_s = ev0.elapsed_time(ev1) / 1e3 / reps
        ph1 = sptt.sptt_batch_phase_ms(b.handle)
        phase_ms = {k: ph1[k] - ph0[k] for k in ph1}  # the timed runs only
    peak, peak_kind = measured_peaks()
    m_s = phase_ms["mttkrp"] / 1e3 / reps  # CTA 0's MTTKRP-phase wall time per run (closing barrier included)
    achieved = sweep_bytes * iters / m_s / 1e9 if m_s > 0 else None
    # one tensor at a time through the single-tensor path (creation not timed)
    cpds = [sptt.Cpd(d, i, v, R, seed=1 + k).init() for k, (d, i, v) in enumerate(tensors)]
    for c in cpds:
        c.iterate(1)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for c in cpds:
        c.iterate(iters)
    ev1.record()
    torch.cuda.synchronize()
    seq_s = ev0.elapsed_time(ev1) / 1e3
    del cpds
    return {"tensors": len(tensors), "total_nnz": int(sum(int(v.numel()) for _, _, v in tensors)),
            "rank": R, "iters": iters, "grid": grid, "chunks_per_mode": chunks[:4], "gen_s": round(gen_s, 1),
            "create_s": round(create_s, 1), "batched_s_per_run": batched_s,
            "plan": {"kind": "batched autotuner (plan 1)", "chosen": {"chunk": sched[0], "variant": sched[2]},
                     "candidates_timed": ncand, "chosen_timed_run_ms": tuned_ms},
            "mttkrp_roofline": {"bound": "hbm", "bytes_per_run": sweep_bytes * iters, "phase_s_per_run": m_s,
                                "achieved": achieved, "peak": peak, "unit": "GB/s",
                                "frac": None if achieved is None else achieved / peak, "peak_kind": peak_kind,
                                "time_source": "CTA 0's MTTKRP-phase wall time (globaltimer), closing barrier "
                                               "included"},
            "phase_ms_timed_runs": phase_ms,
            "batched_GnnzR_per_s": work / batched_s / 1e9, "sequential_s": seq_s,
            "sequential_GnnzR_per_s": work / seq_s / 1e9, "speedup": seq_s / batched_s}


def mixed4_extra(args, dev):
    """The 4-mode mixed-precision workload, 2e6 x 5e5 x 5e4 x 1e3, 1.5e8
    non-zeros, R = 64, from the same initial factors:
      fixed count: 25 BF16 iterations + one FP32 refinement sweep against 26
        FP32 iterations (time of the whole run, the sweep included);
      converged: both run until the fit gains less than 1e-5 per iteration
        (Algorithm 1's stop rule), the mixed run then does its FP32 sweep;
      and 26 FP32 iterations from the same start rounded to BF16 (the fit's
        sensitivity to a BF16-sized change of the start alone).
    Also the BF16 R = 64 MTTKRP's HBM fraction under the byte model."""
    import torch

    import paper_1812_05961_gb300 as sptt
    import tensorgen

    t0 = time.time()
    t = tensorgen.powerlaw4(seed=3, device=dev)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    torch.cuda.empty_cache()
    R = 64
    stream = torch.cuda.current_stream()
    distinct = [int(torch.unique(x).numel()) for x in t.inds]
    out = {"workload": "power-law 4-mode %s, %d nnz, Zipf(1.2), values U(0,1), R=64" %
                       ("x".join(map(str, t.dims)), t.nnz), "gen_s": round(gen_s, 1)}

    def ev():
        return torch.cuda.Event(enable_timing=True)

    for name, prec in (("fp32", sptt.SPTT_F32), ("bf16", sptt.SPTT_BF16)):
        c = sptt.Cpd(t.dims, t.inds, t.vals, R, seed=3, precision=prec, profile=1).init()
        torch.cuda.synchronize()
        c.timers()
        a, b, e = ev(), ev(), ev()
        a.record(stream)
        c.iterate(25)
        b.record(stream)
        if prec == sptt.SPTT_BF16:
            c.refine(1)
        else:
            c.iterate(1)
        e.record(stream)
        torch.cuda.synchronize()
        tm = c.timers()
        fixed_fit = c.fit()[0]
        # the same run continued to the stop rule, then (mixed) one FP32 sweep
        c.init()
        a2, b2 = ev(), ev()
        a2.record(stream)
        done = c.iterate(2000, 1e-5)
        if prec == sptt.SPTT_BF16:
            c.refine(1)
        b2.record(stream)
        torch.cuda.synchronize()
        out[name] = {"s_per_iter": a.elapsed_time(b) / 25 / 1e3, "last_sweep_s": b.elapsed_time(e) / 1e3,
                     "total_26_s": a.elapsed_time(e) / 1e3, "s_per_iter_incl_sweep": a.elapsed_time(e) / 26 / 1e3,
                     "fit_26": fixed_fit,
                     "converged": {"iters": done, "fit": c.fit()[0], "s": a2.elapsed_time(b2) / 1e3},
                     "mttkrp_ms_per_launch": tm["mttkrp"][0] / max(tm["mttkrp"][1], 1),
                     "GnnzR_per_s": 4 * t.nnz * R * 26 / (a.elapsed_time(e) / 1e3) / 1e9}
        if prec == sptt.SPTT_BF16:
            csfs = [sptt.Csf(t.dims, t.inds, t.vals, r) for r in range(4)]
            bpl = sum(byte_model(cs, t.dims, R, distinct, 2) for cs in csfs) / 4
            del csfs
            peak, kind = measured_peaks()
            ach = bpl / (out[name]["mttkrp_ms_per_launch"] * 1e-3) / 1e9
            out[name]["roofline"] = {"bound": "hbm", "bytes_per_launch": int(bpl), "achieved": ach, "peak": peak,
                                     "unit": "GB/s", "frac": ach / peak, "peak_kind": kind}
        del c
        torch.cuda.empty_cache()
    # plain FP32 from the same start rounded to BF16: how far the 26-iteration
    # fit moves under a BF16-sized change of the start alone
    c = sptt.Cpd(t.dims, t.inds, t.vals, R, seed=3).init()
    start = [c.factor(m).to(torch.bfloat16).float() for m in range(len(t.dims))]
    c.init(start)
    c.iterate(26)
    out["fp32_from_bf16_start_fit_26"] = c.fit()[0]
    del c, start
    torch.cuda.empty_cache()
    out["delta_fit_26_fp32_from_bf16_start_vs_fp32"] = out["fp32_from_bf16_start_fit_26"] - out["fp32"]["fit_26"]
    out["delta_fit_26_bf16_vs_fp32_from_bf16_start"] = out["bf16"]["fit_26"] - out["fp32_from_bf16_start_fit_26"]
    out["delta_fit_26_bf16_vs_fp32"] = out["bf16"]["fit_26"] - out["fp32"]["fit_26"]
    out["delta_fit_converged_bf16_vs_fp32"] = out["bf16"]["converged"]["fit"] - out["fp32"]["converged"]["fit"]
    out["speedup_26_bf16_plus_sweep_vs_fp32"] = out["fp32"]["total_26_s"] / out["bf16"]["total_26_s"]
    out["speedup_converged"] = out["fp32"]["converged"]["s"] / out["bf16"]["converged"]["s"]
    del t
    torch.cuda.empty_cache()
    return out


def tiling_extra(args, t, dev):
    """Mode tiling at R = 32 with FP32 gathers on the bench tensor (the
    2,000-row leaf factor is 256 KB, above the 160 KB shared-memory table):
    tiles of as many rows as the table holds against the untiled default;
    s/iter, MTTKRP ms per launch, the HBM fraction under the untiled CSFs'
    byte model (the same MTTKRP work) and the fit after 10 iterations."""
    import torch

    import paper_1812_05961_gb300 as sptt
    R, dims = 32, t.dims
    distinct = [int(torch.unique(x).numel()) for x in t.inds]
    stream = torch.cuda.current_stream()
    orders = [sptt.sptt_level_order(dims, r, sptt.sptt_sched_default(dims, r, R, sptt.SPTT_F32, t.nnz)[3])
              for r in range(3)]
    csfs = [sptt.Csf(dims, t.inds, t.vals, r, level_order=orders[r]) for r in range(3)]
    bpl = sum(byte_model(c, dims, R, distinct, 4) for c in csfs) / 3
    del csfs
    peak, kind = measured_peaks()
    out = {"rank": R, "byte_model_per_launch_untiled": int(bpl)}
    for name, kw in (("untiled", {}), ("tiled", {"leaf_tile_rows": -1})):
        c = sptt.Cpd(dims, t.inds, t.vals, R, seed=1, profile=1, **kw).init()
        c.iterate(2)
        torch.cuda.synchronize()
        c.timers()
        base = c.timers()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c.iterate(8)
        b.record(stream)
        torch.cuda.synchronize()
        tm = c.timers()
        ms = (tm["mttkrp"][0] - base["mttkrp"][0]) / max(tm["mttkrp"][1] - base["mttkrp"][1], 1)
        out[name] = {"s_per_iter": a.elapsed_time(b) / 8 / 1e3, "mttkrp_ms_per_launch": ms,
                     "frac_of_hbm_under_untiled_model": bpl / (ms * 1e-3) / 1e9 / peak, "fit_after_10": c.fit()[0]}
        del c
        torch.cuda.empty_cache()
    out["peak_kind"] = kind
    return out


def mixed_vs_oracle_extra(dev):
    """Mixed precision against the FP64 oracle on a scaled-down 4-mode
    power-law tensor (8,000 x 2,000 x 500 x 100, 3e5 non-zeros, Zipf(1.2),
    R = 64), from the same initial factors: after K = 26 and K = 100
    iterations, the oracle, the FP32 path and the mixed path (K - 1 BF16
    iterations + one FP32 sweep); signed fit differences against the oracle
    and each factor's relative error."""
    import numpy as np

    import oracle
    import paper_1812_05961_gb300 as sptt
    import tensorgen
    dims, nnz, R, seed = (8000, 2000, 500, 100), 300_000, 64, 3
    counts = (26, 100)
    t = tensorgen.sample_unique(dims, nnz, 31, "cpu", dist="zipf", s=1.2, values="uniform")
    inds, vals = t.numpy()
    cores, _ = host_cpu()
    threads = oracle.set_threads(cores)
    t0 = time.time()
    ref = {k: oracle.cpd_als(inds, vals, dims, R, k, seed=seed) for k in counts}
    oracle_s = time.time() - t0
    out = {"workload": "power-law 4-mode 8000x2000x500x100, 3e5 nnz, Zipf(1.2), U(0,1), R=64",
           "oracle": {"threads": threads, "s": round(oracle_s, 1),
                      "fit": {str(k): float(ref[k]["fits"][-1]) for k in counts}}}
    di = [x.to(dev) for x in t.inds]
    dv = t.vals.to(dev)

    def rel(a, b):
        a = a.numpy().astype(np.float64)
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    for k in counts:
        row = {}
        for name, prec in (("fp32", sptt.SPTT_F32), ("mixed", sptt.SPTT_BF16)):
            c = sptt.Cpd(dims, di, dv, R, seed=seed, precision=prec).init()
            if prec == sptt.SPTT_BF16:
                c.iterate(k - 1)
                c.refine(1)
            else:
                c.iterate(k)
            fit = c.fit()[0]
            row[name] = {"fit": fit, "delta_fit_vs_oracle": fit - float(ref[k]["fits"][-1]),
                         "factor_rel_err": [rel(c.factor(m), ref[k]["factors"][m]) for m in range(4)]}
            del c
        out["iters_%d" % k] = row
    return out


def one_csf_extra(args, t, R, dev):
    """One CSF for all modes (the non-root modes by sptt_mttkrp_mode) against
    one CSF per mode, on the bench tensor: per-mode MTTKRP times, CP-ALS
    s/iter, CSF memory and the fit after 10 iterations."""
    import torch

    import paper_1812_05961_gb300 as sptt
    dims = t.dims
    stream = torch.cuda.current_stream()

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    F = [torch.rand(d, R, device=dev) for d in dims]
    out = {}
    for csf_mode in (1, 2):
        root = min(range(3), key=lambda m: (dims[m], m)) if csf_mode == 1 else max(range(3), key=lambda m: (dims[m], -m))
        c = sptt.Csf(dims, t.inds, t.vals, root)
        csf_bytes = sum(n * 4 for n in c.nfibs) + sum(n * 4 for n in c.nfibs[:-1]) + c.nfibs[-1] * 5
        ms = {}
        for m in range(3):
            o = torch.empty(dims[m], R, device=dev)
            ms["mode%d" % m] = timed(lambda: c.mttkrp_mode(m, F, out=o))
            if m != root:
                ms["mode%d_global_only" % m] = timed(lambda: c.mttkrp_mode(m, F, out=o, sched=(128, 256, 1)))
        del c
        cpd = sptt.Cpd(dims, t.inds, t.vals, R, seed=1, csf_mode=csf_mode).init()
        cpd.iterate(2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cpd.iterate(8)
        b.record(stream)
        torch.cuda.synchronize()
        s_iter = a.elapsed_time(b) / 8 / 1e3
        out["csf_mode%d" % csf_mode] = {"root": root, "mttkrp_ms": ms, "s_per_iter": s_iter,
                                        "GnnzR_per_s": 3 * t.nnz * R / s_iter / 1e9, "fit_after_10": cpd.fit()[0],
                                        "csf_bytes": csf_bytes}
        del cpd
        torch.cuda.empty_cache()
    ref = sptt.Cpd(dims, t.inds, t.vals, R, seed=1).init()
    ref.iterate(10)
    out["per_mode_fit_after_10"] = ref.fit()[0]
    del ref
    torch.cuda.empty_cache()
    return out


def sched_extra(args, dev):
    """The learned scheduler the package ships (trained on the GPU by the
    library's MLP kernels on autotuner sweeps of generated tensors; see
    paper_1812_05961_gb300/train_scheduler.py) against the library's fixed
    default rule, on held-out generated tensors of the same distribution
    (other seeds: 1e5-2e7 and 2e7-2e8 non-zeros) and on a 5-mode probe
    tensor; regret = time of the chosen
    schedule over the best one found by the exhaustive autotuner, minus 1."""
    import torch

    from paper_1812_05961_gb300 import schedtrain, train_scheduler
    import tensorgen

    if not os.path.exists(train_scheduler.MODEL):
        return {"unavailable": "no trained model at %s" % os.path.basename(train_scheduler.MODEL)}
    with open(train_scheduler.MODEL) as f:
        meta = json.load(f).get("meta", {})
    model = train_scheduler.load()
    t0 = time.time()
    held = train_scheduler.sweep(train_scheduler.tensor_specs(args.sched_heldout, seed=77), dev)
    held_large = train_scheduler.sweep(train_scheduler.tensor_specs(12, 79, nnz_max=2e8, nnz_min=2e7), dev)
    dims = [1_000_000, 1_000_000, 100_000, 10_000, 500]
    t = tensorgen.sample_unique(dims, 200_000_000, 5, dev, "zipf", s=1.1, values="uniform")
    probe = schedtrain.Dataset(schedtrain.sweep_tensor(t.dims, t.inds, t.vals, 32, reps=3, label="probe"))
    del t
    torch.cuda.empty_cache()
    res = {"model": {k: meta.get(k) for k in ("tensors", "strata", "nnz_range", "split", "samples", "steps",
                                              "loss_first_last")},
           "heldout_tensors": args.sched_heldout, "heldout_samples": len(held.samples),
           "heldout_large_tensors": 12, "heldout_large_samples": len(held_large.samples),
           "sweep_s": round(time.time() - t0, 1)}
    for name, ds in (("heldout", held), ("heldout_large_2e7_2e8", held_large), ("probe_5mode_2e8_r32", probe)):
        res[name] = {"learned": schedtrain.summarize(schedtrain.regret(ds, model)),
                     "default": schedtrain.summarize(schedtrain.regret(ds))}
    return res


def ours(args, rank, world, local):
    import torch

    import paper_1812_05961_gb300 as sptt
    import tensorgen

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    R = args.rank
    t_gen = time.time()
    t = tensorgen.powerlaw3(seed=args.seed + rank, device=dev, nnz=args.nnz)
    torch.cuda.synchronize()
    t_gen = time.time() - t_gen
    dims = t.dims
    nnz = t.nnz
    distinct = [int(torch.unique(x).numel()) for x in t.inds]
    torch.cuda.empty_cache()  # drop the generator's temporaries

    # CSFs (one per root) are built inside the handle; build the same ones
    # here (the level order the handle takes by default) for the byte model
    bf16 = args.precision == "bf16"
    gdt = sptt.SPTT_BF16 if bf16 else sptt.SPTT_F32
    sched = None if (args.variant == 0 and args.chunk == 0) else (args.chunk, 256, args.variant, 0)
    kinds = [sptt.sptt_sched_default(dims, r, R, gdt, nnz)[3] if sched is None else sched[3] for r in range(3)]
    orders = [sptt.sptt_level_order(dims, r, kinds[r]) for r in range(3)]
    csfs = [sptt.Csf(dims, t.inds, t.vals, r, level_order=orders[r]) for r in range(3)]
    s_f = 2 if bf16 else 4
    bytes_per = [byte_model(c, dims, R, distinct, s_f) for c in csfs]
    flops_per = [flop_model(c, R) for c in csfs]
    gather_per = [every_gather_model(c, R, s_f) for c in csfs]
    nfibs = [c.nfibs for c in csfs]
    del csfs

    t_build = time.time()
    cpd = sptt.Cpd(dims, t.inds, t.vals, R, seed=1, profile=1, sched=sched,
                   precision=sptt.SPTT_BF16 if bf16 else sptt.SPTT_F32)
    t_build = time.time() - t_build
    cpd.init()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        cpd.iterate(1)
    torch.cuda.synchronize()
    cpd.timers()  # drain warm-up timer records
    base_timers = cpd.timers()
    l0 = sptt.sptt_debug_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            cpd.iterate(1)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = sptt.sptt_debug_launch_count() - l0
    ms_total = ev0.elapsed_time(ev1)
    tm = cpd.timers()
    mttkrp_ms = tm["mttkrp"][0] - base_timers["mttkrp"][0]
    mttkrp_n = tm["mttkrp"][1] - base_timers["mttkrp"][1]
    routines = {k: (tm[k][0] - base_timers[k][0]) / args.steps for k in tm}
    fit = cpd.fit()[0]
    ms_total = max_over_ranks(ms_total, dist, dev)
    ms_step = ms_total / args.steps
    value = job_rate(3 * nnz * R * args.steps, world, ms_total * 1e-3)

    peak, peak_kind = measured_peaks()
    # MTTKRP routine (zero-fill + kernel) per launch; the three roots differ,
    # so the algorithmic bytes are summed over the modes and divided by the total time
    alg_bytes = sum(bytes_per) * args.steps
    achieved = alg_bytes / (mttkrp_ms * 1e-3) / 1e9
    # measured traffic applies while the timed kernel is the captured one
    traffic = None
    ncu = NCU_TRAFFIC_BF16 if bf16 else NCU_TRAFFIC
    # (the captures are of the kernels the default rule picks from 2^25 non-zeros on)
    if sched is None and R in (16,) and len(dims) == 3 and ncu is not None and nnz >= 2 ** 25:
        traffic = sum(ncu["bytes"]) / 3 * nnz / ncu["nnz"]
    flops_s = sum(flops_per) * args.steps / (mttkrp_ms * 1e-3) / 1e12
    fp32_peak, n_sms, peak_mhz = fp32_peak_tflops(dev)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_source": None if traffic is None else
                "ncu dram__bytes_read.sum + dram__bytes_write.sum of %s at %d nnz, scaled by nnz (mean of the 3 roots)"
                % (ncu["kernel"], ncu["nnz"]),
                "every_gather_bytes_per_launch": [int(b) for b in gather_per],
                "fp32_fma": {"achieved_tflops": flops_s, "peak_tflops": fp32_peak,
                             "frac": flops_s / fp32_peak,
                             "peak_kind": "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (n_sms, peak_mhz)},
                "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "bytes_per_launch": [int(b) for b in bytes_per],
                "flops_per_launch": [int(f) for f in flops_per],
                "avg_launch_ms": mttkrp_ms / max(mttkrp_n, 1),
                "launches": mttkrp_n}

    # e2e: the one-shot call from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        h_inds = [x.cpu().pin_memory() for x in t.inds]
        h_vals = t.vals.cpu().pin_memory()
        h_out = [torch.empty(d, R).pin_memory() for d in dims]
        h_lam = torch.empty(R, dtype=torch.float64).pin_memory()
        prec = sptt.SPTT_BF16 if bf16 else sptt.SPTT_F32
        sptt.sptt_cpd_als(dims, h_inds, h_vals, R, 1, factors_out=h_out, lambda_out=h_lam, seed=1, precision=prec)
        torch.cuda.synchronize()
        times = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            sptt.sptt_cpd_als(dims, h_inds, h_vals, R, args.e2e_iters, factors_out=h_out,
                              lambda_out=h_lam, seed=1, precision=prec)
            times.append(time.perf_counter() - t0)
        e2e_t = sum(times) / len(times)
        e2e_t = max_over_ranks(e2e_t, dist, dev)
        h2d = sum(x.numel() * 4 for x in h_inds) + h_vals.numel() * 4
        d2h = sum(d * R * 4 for d in dims) + R * 8 + 8
        e2e = {"value": job_rate(3 * nnz * R * args.e2e_iters, world, e2e_t), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "seconds_per_call": e2e_t, "als_iters_per_call": args.e2e_iters,
               "fp32_refinement_sweeps_per_call": 1 if bf16 else 0}
        del h_inds, h_vals

    extras = {}
    want = set() if args.no_extras else set(x.strip() for x in args.extras.split(",") if x.strip())
    if "precision" in want:
        # mixed precision vs FP32 at the same start, plus rank 32: 20
        # iterations each; the mixed run's last iteration is its FP32
        # refinement sweep, and its time is counted
        res = {}
        for name, prec, r in (("fp32_r16", sptt.SPTT_F32, R), ("bf16_r16", sptt.SPTT_BF16, R),
                              ("fp32_r32", sptt.SPTT_F32, 32), ("bf16_r32", sptt.SPTT_BF16, 32)):
            c = sptt.Cpd(dims, t.inds, t.vals, r, seed=1, precision=prec).init()
            c.iterate(1)  # warm-up: the first call of each precision captures its graph
            if prec == sptt.SPTT_BF16:
                c.refine(1)
            c.init()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if prec == sptt.SPTT_BF16:
                c.iterate(19)
                c.refine(1)
            else:
                c.iterate(20)
            b.record(stream)
            torch.cuda.synchronize()
            s_iter = a.elapsed_time(b) / 20 / 1e3
            res[name] = {"s_per_iter": s_iter, "fit_after_20": c.fit()[0],
                         "GnnzR_per_s": 3 * nnz * r / s_iter / 1e9,
                         "note": "20 iterations timed from the initial factors" +
                                 (", the last one the FP32 refinement sweep" if prec == sptt.SPTT_BF16 else "")}
            del c
        for r in (16, 32):
            f32, b16 = res["fp32_r%d" % r], res["bf16_r%d" % r]
            b16["delta_fit_vs_fp32"] = b16["fit_after_20"] - f32["fit_after_20"]
            b16["speedup_vs_fp32"] = f32["s_per_iter"] / b16["s_per_iter"]
        extras["precision_and_rank"] = res

    if "batched" in want and rank == 0:
        del cpd
        torch.cuda.empty_cache()
        extras["batched"] = batched_extra(args, dev)
    if "sched" in want and rank == 0:
        torch.cuda.empty_cache()
        extras["scheduler"] = sched_extra(args, dev)
    if "tiling" in want and rank == 0:
        torch.cuda.empty_cache()
        extras["tiling"] = tiling_extra(args, t, dev)
    if args.extra_one_csf:
        torch.cuda.empty_cache()
        extras["one_csf"] = one_csf_extra(args, t, R, dev)
    if "mixed4" in want and rank == 0:
        torch.cuda.empty_cache()
        extras["mixed_precision_4mode"] = mixed4_extra(args, dev)
    if "mixed_vs_oracle" in want and rank == 0 and world == 1:
        torch.cuda.empty_cache()
        extras["mixed_vs_oracle"] = mixed_vs_oracle_extra(dev)

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        ci = [x.cpu().numpy() for x in t.inds]
        cv = t.vals.cpu().numpy()
        cores, model = host_cpu()
        threads = oracle.set_threads(cores)
        rate, secs, s = cpu_oracle_rate(ci, cv, dims, R, args.cpu_seconds, threads)
        cpu_base = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                    "host_cores": cores, "cpu_model": model,
                    "sample": "one CP-ALS iteration (3 MTTKRPs + solve + fit) of the FP64 C oracle on "
                              "the first %d of the %d non-zeros, %d threads, %.1f s" % (s, nnz, threads, secs)}

    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32" if bf16 else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rank": R, "step": "one CP-ALS iteration (3 mode updates + fit)",
                       "factor_gathers": "bf16 (fp32 accumulate, fp64 solve)" if bf16 else "fp32",
                       "mttkrp_sched": "default" if sched is None else list(sched),
                       "l2": "inputs larger than L2 (CSF about 0.8 GB per mode)",
                       "parallelism": "replicas" if world > 1 else "single",
                       "nfibs_per_root": nfibs, "level_orders": orders,
                       "gen_s": round(t_gen, 1), "cpd_create_s": round(t_build, 2),
                       "input_checksum": input_checksum(t)},
            "roofline": roofline, "cpu_baseline": cpu_base, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "routines_ms_per_iter": routines, "fit": fit, "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    ours(args, rank, world, local)


if __name__ == "__main__":
    main()
