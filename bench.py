#!/usr/bin/env python3
"""Benchmark of exact planted (l,d)-motif search on one GB300 (or N, one process each).

Default workload: one plain PMS instance per step, (l, d) = (15, 4), n = 20
DNA sequences of length m = 600 (i.i.d. uniform bases, one motif planted in
each sequence with exactly d substitutions), a different seeded instance each
step. `value` is solves/s with the inputs already in device memory, timed
with CUDA events on the library's stream, L2 flushed between steps (outside
the timed events). `e2e` times the host-buffer C-ABI call (pms_solve):
upload, all kernels and the download of the result inside the clock.

Other workloads (--workload): plain9_2, plain17_5, plain19_6 (single
instances), quorum15_4_q10 (the quorum form), protein9_3 / protein9_4 (the
general-alphabet search over the twenty amino acids, n = 20, m = 600,
through the host-buffer call pms_solve_sigma: `value` from the device time
of its kernels, `e2e` from the call's wall time), batch (256 mixed instances
in one persistent launch, compared with the same instances one by one),
serve (Poisson request stream).
`--impl reference` times the CPU oracle on bounded samples instead.
Under torchrun each rank solves its own instances (no data exchange); the
line reports the max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import planted_inputs as pi  # noqa: E402

METRIC = "PMS solves/s and candidate checks/s per (l,d); batched/served vs plain, 1 GB300"
WORKLOADS = {
    "plain9_2": (9, 2), "plain15_4": (15, 4), "plain17_5": (17, 5), "plain19_6": (19, 6),
}
# quorum form: (l, d, q), n = 20, m = 600
QUORUM_WORKLOADS = {"quorum15_4_q10": (15, 4, 10)}
# general alphabet, the twenty amino acids: (l, d), n = 20, m = 600
PROTEIN_WORKLOADS = {f"protein{l}_{d}": (l, d) for (l, d) in pi.PROTEIN_LD}
L2_FLUSH_BYTES = 512 << 20

# DRAM bytes (read + write) per launch of the verification kernel from one ncu
# capture (profiles/main_kernel_plain*.md), valid only for the kernel source
# they were taken on (its sha256 prefix); otherwise the bench reports null.
NCU_TRAFFIC = {"kernel_sha256": "c1cb4e4a809d7da7", "plain15_4": 1.080064e6, "plain17_5": 1.095680e6}


def kernel_sha() -> str:
    import hashlib
    with open(os.path.join(ROOT, "paper_2403_00306_gb300", "csrc", "pms_kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_traffic(workload: str):
    if kernel_sha() != NCU_TRAFFIC["kernel_sha256"]:
        return None
    return NCU_TRAFFIC.get(workload)


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:  # noqa: BLE001
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"pms_bench_clocks_{os.getpid()}_rank{index}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict | None:
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws: int):
    if ws <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group("gloo")
    return dist


def max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def rank_seeds(rank: int, count: int, base: int = 1) -> list[int]:
    """Instance seeds of one rank: ranks solve disjoint instances (weak scaling, no data exchange)."""
    return [base + rank * 100000 + i for i in range(count)]


def n_ball(l: int, d: int, sigma: int = 4) -> int:
    return sum(math.comb(l, i) * (sigma - 1) ** i for i in range(d + 1))


# ------------------------------------------------------------------ CPU baseline (oracle)

def cpu_oracle_rate(l: int, d: int, n: int, m: int, seed: int, budget_s: float, q: int = 0,
                    alphabet: bytes | None = None) -> dict:
    """The oracle as it stands, on a bounded slice of seeds of one instance, scaled to solves/s
    (q > 0: the quorum form, seeds over s_1 .. s_{n-q+1}; alphabet: the general-alphabet search)."""
    import oracle
    o = oracle.Oracle()
    inst = pi.planted_instance_sigma(n, m, l, d, seed, alphabet) if alphabet else pi.planted_instance(n, m, l, d, seed)
    W = (m - l + 1) * (n - q + 1 if q > 0 else 1)
    cores = os.cpu_count() or 1
    sigma = len(alphabet) if alphabet else 4

    def run(lo, hi):
        if alphabet:
            o.sigma_solve_seeds(inst.seqs, l, d, alphabet, lo, hi, q=q, threads=cores)
        elif q > 0:
            o.solve_quorum_seeds(inst.seqs, l, d, q, lo, hi, threads=cores)
        else:
            o.solve_seeds(inst.seqs, l, d, lo, hi, threads=cores)

    # calibrate on one seed per core, then grow to about budget_s
    k = min(W, cores)
    t0 = time.perf_counter()
    run(0, k)
    t1 = time.perf_counter() - t0
    total_t, total_seeds, lo = t1, k, k
    while total_t < budget_s and lo < W:
        per_seed = max(total_t / total_seeds, 1e-6)
        take = int(min(W - lo, max(cores, (budget_s - total_t) / per_seed)))
        take = max(1, take)
        t0 = time.perf_counter()
        run(lo, lo + take)
        total_t += time.perf_counter() - t0
        total_seeds += take
        lo += take
    solves_per_s = (total_seeds / W) / total_t
    return {"value": solves_per_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{total_seeds} of {W} seeds of one ({l},{d}{f',q={q}' if q else ''}) n={n} m={m} "
                      f"{'protein ' if alphabet else ''}instance, {total_t:.1f} s, scaled by {W}/{total_seeds}",
            "candidate_checks_per_s": total_seeds * n_ball(l, d, sigma) / total_t}


def run_reference(args, ws, rank) -> None:
    if rank != 0:
        return
    alphabet = pi.PROTEIN if args.workload in PROTEIN_WORKLOADS else None
    if alphabet:
        (l, d), q = PROTEIN_WORKLOADS[args.workload], 0
    else:
        l, d, q = QUORUM_WORKLOADS[args.workload] if args.workload in QUORUM_WORKLOADS \
            else (*WORKLOADS.get(args.workload, (15, 4)), 0)
    n, m = 20, 600
    budget = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for s in range(args.warmup):
        cpu_oracle_rate(l, d, n, m, 1000 + s, budget / 4, q=q, alphabet=alphabet)
    rates = []
    for s in range(args.steps):
        rates.append(cpu_oracle_rate(l, d, n, m, 1 + s, budget, q=q, alphabet=alphabet))
    value = statistics.mean(r["value"] for r in rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": (f"quorum ({l},{d}) q={q}" if q else
                                    f"protein ({l},{d})" if alphabet else f"plain ({l},{d})")
                                   + f" n={n} m={m}, CPU oracle on bounded seed samples"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": rates[0]["cores"], "kind": "oracle",
                             "sample": rates[0]["sample"]},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arms

def make_flush(torch, dev):
    buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def flush(i):
        buf.fill_(i)
    return flush


def bench_plain(args, ws, rank, local, dist, l, d, q: int = 0) -> dict:
    import torch
    import paper_2403_00306_gb300 as pms
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n, m = 20, 600
    K, Wm = args.steps, args.warmup
    seeds = rank_seeds(rank, K + Wm)
    insts = [pi.planted_instance(n, m, l, d, s) for s in seeds]
    d_in = [torch.from_numpy(i.seqs.copy()).to(dev) for i in insts]
    cap = 1 << 16
    d_out = torch.zeros(cap, dtype=torch.int64, device=dev)
    d_st = torch.zeros(4, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = pms.Context(local)
    ctx.set_stream(stream)
    if q:
        ctx.set_options(quorum=q)
    flush = make_flush(torch, dev)

    # parity spot-check of the timed launch configuration against the host path
    ref = ctx.solve(insts[0].seqs, l, d)
    with torch.cuda.stream(stream):
        ctx.solve_device(d_in[0], n, m, l, d, d_out, cap, d_st)
    stream.synchronize()
    st = d_st.cpu().numpy().astype(np.uint32)
    assert st[2] == 0 and np.array_equal(d_out[: st[1]].cpu().numpy().astype(np.uint64), ref), "device path mismatch"

    for i in range(Wm):
        with torch.cuda.stream(stream):
            ctx.solve_device(d_in[i], n, m, l, d, d_out, cap, d_st)
    stream.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    verify_ms = []
    barrier(dist)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(K):
            with torch.cuda.stream(stream):
                flush(k)
                ev[k][0].record(stream)
                ctx.solve_device(d_in[Wm + k], n, m, l, d, d_out, cap, d_st)
                ev[k][1].record(stream)
            verify_ms.append(ctx.stats()["ms_verify"])   # waits for this step's kernels
        torch.cuda.synchronize(dev)
    barrier(dist)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    local_total = sum(step_ms)
    total_ms = max_over_ranks(dist, local_total)
    solves = sum_over_ranks(dist, K)
    value = solves / (total_ms / 1000.0)

    # algorithmic work of the dominant kernel (count mode, same instances, untimed)
    cctx = pms.Context(local)
    cctx.set_options(count_work=1, quorum=q)
    cmp_total = 0
    tested = 0
    for k in range(K):
        cctx.solve(insts[Wm + k].seqs, l, d)
        s = cctx.stats()
        # comparisons of the verification kernel only (the (n - 1) W^2 of the
        # compatibility masks are another kernel's)
        cmp_total += s["cmp_reduce"] + s["cmp_verify"]
        tested += s["candidates_tested"]
    cctx.close()
    cmp_per_launch = cmp_total / K
    verify_avg_ms = statistics.mean(verify_ms)

    # e2e through the host-buffer C-ABI call
    e2e_ms = []
    torch.cuda.synchronize(dev)
    for k in range(K):
        flush(k)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.solve(insts[Wm + k].seqs, l, d)
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
    e2e_total = max_over_ranks(dist, sum(e2e_ms))
    e2e_value = solves / (e2e_total / 1000.0)

    probe = ctx.probe_int_rate(3)   # comparisons per clock per SM (measured)
    probe_popc = ctx.probe_int_rate(0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = load_peaks()
    fmax = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_cmp = probe * sms * fmax
    achieved = cmp_per_launch / (verify_avg_ms / 1000.0) if verify_avg_ms > 0 else float("nan")
    clocks = clk.summary()
    ctx.close()
    W = m - l + 1
    return {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": K, "warmup": Wm,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": (f"quorum ({l},{d}) q={q}" if q else f"plain ({l},{d})")
                               + f" n={n} m={m}, one seeded FM-model instance per step",
                   "l": l, "d": d, "n": n, "m": m, "l2": "flushed between steps (512 MiB write, untimed)",
                   "timing": "CUDA events on the library stream around pms_solve_device"},
        "candidate_checks_per_s": solves * W * (n - q + 1 if q else 1) * n_ball(l, d) / (total_ms / 1000.0),
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_cmp / 1e12,
                     "unit": "Tcmp/s", "frac": achieved / peak_cmp,
                     "traffic": measured_traffic(f"quorum{l}_{d}_q{q}" if q else f"plain{l}_{d}"),
                     "kernel": "main_kernel (verification)", "cmp_per_launch": cmp_per_launch,
                     "verify_ms_per_launch": verify_avg_ms,
                     "peak_basis": f"{probe:.2f} comparisons/clk/SM (probe) x {sms} SMs x {fmax/1e6:.0f} MHz; "
                                   f"POPC probe {probe_popc:.2f}/clk/SM",
                     "share_of_step": verify_avg_ms / (total_ms / K)},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": n * m,
                "d2h_bytes_per_step": 16 + 512 * 8, "ms_per_step": e2e_total / K},
        "gpu_launches": 3 * K,   # packing + compatibility masks, verification, sort/unique
        "clocks": clocks,
        "candidates_tested_per_step": tested / K,
    }


def bench_sigma(args, ws, rank, local, dist, l, d) -> dict:
    """The general-alphabet search on protein instances through pms_solve_sigma (host buffers)."""
    import torch
    import paper_2403_00306_gb300 as pms
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n, m = 20, 600
    K, Wm = args.steps, args.warmup
    seeds = rank_seeds(rank, K + Wm)
    insts = [pi.planted_instance_sigma(n, m, l, d, s) for s in seeds]
    stream = torch.cuda.Stream(device=dev)
    ctx = pms.Context(local)
    ctx.set_stream(stream)
    flush = make_flush(torch, dev)
    for i in range(Wm):
        ctx.solve_sigma(insts[i].seqs, l, d, pi.PROTEIN)
    kern_ms, verify_ms, e2e_ms, cmps = [], [], [], []
    barrier(dist)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(K):
            with torch.cuda.stream(stream):
                flush(k)
            stream.synchronize()
            t0 = time.perf_counter()
            out = ctx.solve_sigma(insts[Wm + k].seqs, l, d, pi.PROTEIN)
            e2e_ms.append((time.perf_counter() - t0) * 1000.0)
            s = ctx.stats()
            kern_ms.append(s["ms_kernel"])
            verify_ms.append(s["ms_verify"])
            # one POPC per comparison: window vs seed, node bound, candidate vs row
            cmps.append(s["cmp_rows"] + s["cmp_reduce"] + s["cmp_verify"])
            assert insts[Wm + k].motif in {bytes(r) for r in out}, "planted motif missing"
        torch.cuda.synchronize(dev)
    barrier(dist)
    total_ms = max_over_ranks(dist, sum(kern_ms))
    solves = sum_over_ranks(dist, K)
    value = solves / (total_ms / 1000.0)
    e2e_total = max_over_ranks(dist, sum(e2e_ms))
    probe_popc = ctx.probe_int_rate(0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = load_peaks()
    fmax = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak = probe_popc * sms * fmax
    verify_avg = statistics.mean(verify_ms)
    achieved = statistics.mean(cmps) / (verify_avg / 1000.0) if verify_avg > 0 else float("nan")
    clocks = clk.summary()
    ctx.close()
    W = m - l + 1
    return {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": K, "warmup": Wm,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"protein ({l},{d}) n={n} m={m}, 20-letter alphabet, one seeded FM-model "
                               f"instance per step", "l": l, "d": d, "n": n, "m": m, "sigma": 20,
                   "l2": "flushed between steps (512 MiB write, untimed)",
                   "timing": "CUDA events on the library stream from the packing kernel to the sort kernel"},
        "candidate_checks_per_s": solves * W * n_ball(l, d, 20) / (total_ms / 1000.0),
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tcmp/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "sigma_main_kernel (search)",
                     "cmp_per_launch": statistics.mean(cmps), "verify_ms_per_launch": verify_avg,
                     "peak_basis": f"one POPC per comparison: {probe_popc:.2f} POPC/clk/SM (probe) x {sms} SMs x "
                                   f"{fmax/1e6:.0f} MHz",
                     "share_of_step": verify_avg / (total_ms / K)},
        "e2e": {"value": solves / (e2e_total / 1000.0), "unit": "solves/s", "h2d_bytes_per_step": n * m,
                "d2h_bytes_per_step": 32 + 8 * 9 + l, "ms_per_step": e2e_total / K},
        "gpu_launches": 3 * K,   # packing, search, sort/unique
        "clocks": clocks,
    }


def bench_batch(args, ws, rank, local, dist) -> dict:
    import torch
    import paper_2403_00306_gb300 as pms
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    insts = pi.batch_instances(count=256, master_seed=2024 + rank)
    ctx = pms.Context(local)
    batch = [(i.seqs, i.l, i.d) for i in insts]
    t_tune = time.perf_counter()
    ctx.set_options(autotune=1)      # tunes each (l, d, n, m) class once, untimed
    ctx.solve_batch(batch)
    t_tune = time.perf_counter() - t_tune
    for _ in range(args.warmup):
        ctx.solve_batch(batch)
    flush = make_flush(torch, dev)
    barrier(dist)
    ts = []
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush(k)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            res = ctx.solve_batch(batch)
            ts.append(time.perf_counter() - t0)
    barrier(dist)
    one = []
    for k in range(max(1, args.steps // 2)):
        t0 = time.perf_counter()
        for i in insts:
            ctx.solve(i.seqs, i.l, i.d)
        one.append(time.perf_counter() - t0)
    total = max_over_ranks(dist, sum(ts))
    solves = sum_over_ranks(dist, 256 * args.steps)
    value = solves / total
    cand = sum((i.m - i.l + 1) * n_ball(i.l, i.d) for i in insts)
    ok = all(not isinstance(r, Exception) for r in res)
    ctx.close()
    return {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "batch of 256 instances, (l,d) in {(11,3),(13,4),(15,4)}, n in [10,30], m in [300,1000]",
                       "timing": "host clock around pms_solve_batch (upload, kernels, download)"},
            "candidate_checks_per_s": cand * args.steps / sum(ts),
            "one_by_one_solves_per_s": 256 / statistics.mean(one), "all_ok": ok, "autotune_s": t_tune,
            "e2e": {"value": value, "unit": "solves/s",
                    "h2d_bytes_per_step": int(sum(i.n * i.m for i in insts)), "d2h_bytes_per_step": None},
            "gpu_launches": 4 * args.steps, "clocks": clk.summary()}


def bench_serve(args, ws, rank, local, dist) -> dict:
    """Poisson request stream through the served form (continuous batching)."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    import torch
    import paper_2403_00306_gb300 as pms
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    count, rate = args.serve_requests, args.serve_rate
    reqs = list(pi.serve_requests(count=count, rate_per_s=rate, master_seed=7 + rank))
    ctx = pms.Context(local)
    # warm-up: a few requests, not timed
    for _, inst in reqs[: max(3, args.warmup)]:
        ctx.wait(ctx.submit(inst.seqs, inst.l, inst.d))
    lat = [None] * count
    done_t = [None] * count
    ok = [True] * count
    pool = ThreadPoolExecutor(max_workers=128)
    lock = threading.Lock()

    def waiter(i, t, arrival):
        try:
            ctx.wait(t)
        except Exception:  # noqa: BLE001
            ok[i] = False
        now = time.perf_counter()
        with lock:
            done_t[i] = now
            lat[i] = now - arrival
        ctx.release(t)

    barrier(dist)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        futs = []
        for i, (ta, inst) in enumerate(reqs):
            target = t0 + ta
            delay = target - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            arrival = max(target, time.perf_counter()) if delay <= 0 else target
            t = ctx.submit(inst.seqs, inst.l, inst.d)
            futs.append(pool.submit(waiter, i, t, arrival))
        for f in futs:
            f.result()
        t_end = max(done_t)
    pool.shutdown()
    st = ctx.stats()
    # saturation: all requests of a slice submitted at once
    sat_n = min(count, 2000)
    ts = time.perf_counter()
    tickets = [ctx.submit(inst.seqs, inst.l, inst.d) for _, inst in reqs[:sat_n]]
    for t in tickets:
        ctx.wait(t)
        ctx.release(t)
    sat = sat_n / (time.perf_counter() - ts)
    ctx.close()
    span = t_end - t0
    solves = sum_over_ranks(dist, count)
    span_max = max_over_ranks(dist, span)
    lat_ms = sorted(1000.0 * x for x in lat)
    cand = sum((inst.m - inst.l + 1) * n_ball(inst.l, inst.d) for _, inst in reqs)
    return {"metric": METRIC, "value": solves / span_max, "unit": "solves/s", "n_gpus": ws, "steps": count,
            "warmup": args.warmup, "ms_per_step": 1000.0 * span_max / count, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"served: {count} Poisson requests at {rate}/s, (l,d) in {{(13,4),(15,4),(17,5)}}, "
                                   "n=20, m in [200,1200]",
                       "timing": "host clock from each arrival to pms_wait's return"},
            "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[int(len(lat_ms) * 0.99) - 1],
                           "max": lat_ms[-1]},
            "offered_per_s": rate, "saturation_solves_per_s": sat,
            "candidate_checks_per_s": cand / span, "all_ok": all(ok),
            "serve": {"waves": st["serve_waves"], "overlapped_waves": st["serve_overlapped_waves"],
                      "max_requests_per_wave": st["serve_max_requests_per_wave"]},
            "e2e": {"value": solves / span_max, "unit": "solves/s",
                    "h2d_bytes_per_step": int(statistics.mean(i.n * i.m for _, i in reqs)),
                    "d2h_bytes_per_step": 16 + 512 * 8},
            "gpu_launches": 3 * count + int(st["serve_waves"]), "clocks": clk.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="plain15_4",
                    choices=sorted(WORKLOADS) + sorted(QUORUM_WORKLOADS) + sorted(PROTEIN_WORKLOADS)
                    + ["batch", "serve"])
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    ws, rank, local = dist_env()
    dist = init_dist(ws)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "batch":
        line = bench_batch(args, ws, rank, local, dist)
    elif args.workload == "serve":
        line = bench_serve(args, ws, rank, local, dist)
    elif args.workload in PROTEIN_WORKLOADS:
        l, d = PROTEIN_WORKLOADS[args.workload]
        line = bench_sigma(args, ws, rank, local, dist, l, d)
        if rank == 0 and ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_rate(l, d, 20, 600, 424242, budget_s=15.0, alphabet=pi.PROTEIN)
    else:
        l, d, q = QUORUM_WORKLOADS[args.workload] if args.workload in QUORUM_WORKLOADS else (*WORKLOADS[args.workload], 0)
        line = bench_plain(args, ws, rank, local, dist, l, d, q)
        if rank == 0 and ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_rate(l, d, 20, 600, 424242, budget_s=15.0, q=q)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
