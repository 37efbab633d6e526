#!/usr/bin/env python3
"""Benchmark of exact planted (l,d)-motif search on one GB300 (or N, one process each).

Default workload: one plain PMS instance per step, (l, d) = (15, 4), n = 20
DNA sequences of length m = 600 (i.i.d. uniform bases, one motif planted in
each sequence with exactly d substitutions), a different seeded instance each
step. `value` is solves/s with the inputs already in device memory, timed
with CUDA events on the library's stream, L2 flushed between steps (outside
the timed events). `e2e` times the host-buffer C-ABI call (pms_solve):
the transfer of the input from pinned host memory, all kernels and the
transfer of the result back inside the clock (for small inputs and
results, such as these, the kernels read and write the pinned host buffers
directly).

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

# DRAM bytes (read + write) per launch of each search kernel from one-pass ncu
# captures (dram__bytes_read.sum + dram__bytes_write.sum, profiles/*.md), valid
# only for the sources they were taken on (sha256 prefix of the kernel file and
# the shared header); otherwise the bench reports null.
NCU_TRAFFIC = {
    "pms_kernels.cu": {"sha256": "74f437207a783ca1+69100b3a5b5aee1d",
                       "plain9_2": 1.099520e6, "plain15_4": 1.066240e6,
                       "plain17_5": 1.102336e6, "plain19_6": 1.618432e6},
    "pms_sigma.cu": {"sha256": "f08996edcfffd0da+69100b3a5b5aee1d", "protein9_4": 4.6230528e7},
}

def source_sha(name: str) -> str:
    import hashlib
    csrc = os.path.join(ROOT, "paper_2403_00306_gb300", "csrc")
    parts = []
    for f in (name, "pms_internal.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            parts.append(hashlib.sha256(fh.read()).hexdigest()[:16])
    return "+".join(parts)


def measured_traffic(source: str, workload: str):
    entry = NCU_TRAFFIC[source]
    if source_sha(source) != entry["sha256"]:
        return None
    return entry.get(workload)


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

def _oracle():
    import oracle
    return oracle.Oracle()


def cpu_oracle_whole(l: int, d: int, n: int, m: int, seed: int, threads: int) -> dict:
    """One whole solve of one seeded instance by the oracle as it stands (char-level motif test)."""
    o = _oracle()
    inst = pi.planted_instance(n, m, l, d, seed)
    t0 = time.perf_counter()
    motifs = o.solve(inst.seqs, l, d, threads=threads)
    t = time.perf_counter() - t0
    return {"seconds": t, "motifs": int(len(motifs)), "value": 1.0 / t}


def cpu_oracle_slice(l: int, d: int, n: int, m: int, seed: int, budget_s: float, threads: int,
                     variant: str = "seeds", q: int = 0, alphabet: bytes | None = None) -> dict:
    """The oracle on a bounded slice of the seeds of one instance, timed and scaled to solves/s
    (variant "seeds": candidates B(x, d) over the l-mers x of s_1 (of s_1..s_{n-q+1} with a quorum);
    "pairs": the Observation 3.3 pair form; alphabet: the general-alphabet search)."""
    o = _oracle()
    inst = pi.planted_instance_sigma(n, m, l, d, seed, alphabet) if alphabet else pi.planted_instance(n, m, l, d, seed)
    W = (m - l + 1) * (n - q + 1 if q > 0 else 1)

    def run(lo, hi):
        if alphabet:
            o.sigma_solve_seeds(inst.seqs, l, d, alphabet, lo, hi, q=q, threads=threads)
        elif q > 0:
            o.solve_quorum_seeds(inst.seqs, l, d, q, lo, hi, threads=threads)
        elif variant == "pairs":
            o.solve_pairs_seeds(inst.seqs, l, d, lo, hi, threads=threads)
        else:
            o.solve_seeds(inst.seqs, l, d, lo, hi, threads=threads)

    k = min(W, threads)
    t0 = time.perf_counter()
    run(0, k)
    total_t, total_seeds, lo = time.perf_counter() - t0, k, k
    while total_t < budget_s and lo < W:
        per_seed = max(total_t / total_seeds, 1e-6)
        take = max(1, int(min(W - lo, max(threads, (budget_s - total_t) / per_seed))))
        t0 = time.perf_counter()
        run(lo, lo + take)
        total_t += time.perf_counter() - t0
        total_seeds += take
        lo += take
    return {"value": (total_seeds / W) / total_t, "unit": "solves/s", "threads": threads, "seconds": total_t,
            "sample": f"seeds 0..{total_seeds - 1} of the {W} of one {'protein ' if alphabet else ''}"
                      f"({l},{d}{f',q={q}' if q else ''}) n={n} m={m} instance ({variant} form), "
                      f"{total_t:.1f} s, rate scaled by {W}/{total_seeds}"}


def cpu_baseline_plain(l: int, d: int, n: int = 20, m: int = 600, seed: int = 424242) -> dict:
    """cpu_baseline of a plain configuration. (9,2), (15,4): one whole solve on every host core,
    plus a single-thread seed slice. (17,5), (19,6): a whole char-level solve takes tens of
    minutes (about 35 s of one core per seed at (17,5)), so the timed baseline is the oracle's
    Observation 3.3 pair form on one seed per host core, scaled to solves/s."""
    cores = os.cpu_count() or 1
    out = {"unit": "solves/s", "cores": cores, "kind": "oracle"}
    if (l, d) in ((9, 2), (15, 4)):
        w = cpu_oracle_whole(l, d, n, m, seed, cores)
        out.update(value=w["value"], threads=cores,
                   sample=f"one whole ({l},{d}) n={n} m={m} instance (seed {seed}), {w['seconds']:.1f} s on "
                          f"{cores} threads, {w['motifs']} motifs")
        st = cpu_oracle_slice(l, d, n, m, seed, 4.0, 1)
        out["single_thread"] = {"value": st["value"], "unit": "solves/s", "threads": 1, "sample": st["sample"]}
    else:
        pr = cpu_oracle_slice(l, d, n, m, seed, 1.0, cores, variant="pairs")
        out.update(value=pr["value"], threads=cores, sample=pr["sample"],
                   note="char-level seed form not timed here: tens of seconds of one core per seed")
    return out


def run_reference(args, ws, rank) -> None:
    """The reference arm: the CPU oracle as it stands. Plain workloads: each step is one whole
    solve of a new seeded instance on every host core; --steps is honoured as a cap, so that the
    run ends within about two minutes; warm-up steps are 16-seed slices (untimed)."""
    if rank != 0:
        return
    alphabet = pi.PROTEIN if args.workload in PROTEIN_WORKLOADS else None
    if alphabet:
        (l, d), q = PROTEIN_WORKLOADS[args.workload], 0
    else:
        l, d, q = QUORUM_WORKLOADS[args.workload] if args.workload in QUORUM_WORKLOADS \
            else (*WORKLOADS.get(args.workload, (15, 4)), 0)
    n, m = 20, 600
    cores = os.cpu_count() or 1
    o = _oracle()
    for s in range(args.warmup):
        inst = pi.planted_instance(n, m, l, d, 1000 + s)
        if not alphabet and not q:
            o.solve_seeds(inst.seqs, l, d, 0, 16, threads=cores)
    whole = not alphabet and not q and (l, d) in ((9, 2), (15, 4))
    times, fracs, samples = [], [], []
    budget = 120.0
    t_start = time.perf_counter()
    for k in range(args.steps):
        if whole:
            w = cpu_oracle_whole(l, d, n, m, 1 + k, cores)
            times.append(w["seconds"])
            fracs.append(1.0)
            samples.append(f"seed {1 + k}: {w['seconds']:.1f} s, {w['motifs']} motifs")
        else:
            sl = cpu_oracle_slice(l, d, n, m, 1 + k, 15.0, cores, q=q, alphabet=alphabet)
            times.append(sl["seconds"])
            fracs.append(sl["value"] * sl["seconds"])      # the fraction of one solve this step did
            samples.append(sl["sample"])
        elapsed = time.perf_counter() - t_start
        if elapsed + elapsed / (k + 1) > budget:
            break
    steps = len(times)
    value = sum(fracs) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": steps, "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(times) / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": (f"quorum ({l},{d}) q={q}" if q else
                                    f"protein ({l},{d})" if alphabet else f"plain ({l},{d})")
                                   + f" n={n} m={m}, CPU oracle"
                                   + (", one whole solve per step" if whole else ", a bounded seed slice per step"),
                       "steps_note": "--steps is a cap: steps stop once about 120 s have been spent"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "threads": cores, "sample": "; ".join(samples)},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arms

def make_flush(torch, dev):
    buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def flush(i):
        buf.fill_(i)
    return flush


class Peaks:
    """Roofline denominators of the comparison-bound kernels (l-mer comparisons per second)."""

    def __init__(self, ctx, torch, dev):
        self.popc = ctx.probe_int_rate(0)       # POPC per clock per SM (measured probe)
        self.mix = ctx.probe_int_rate(3)        # the comparison mix per clock per SM (measured probe)
        self.sms = torch.cuda.get_device_properties(dev).multi_processor_count
        self.fmax = float(load_peaks().get("sm_max_mhz", 2070.0)) * 1e6
        self.peak_popc = self.popc * self.sms * self.fmax
        # 4 integer issue slots per comparison (2 LOP3, POPC, IMNMX) on 128 lanes per SM
        self.peak_int4 = self.sms * 128 * self.fmax / 4.0

    def roofline(self, cmp_per_launch: float, ms: float, kernel: str, traffic, share: float) -> dict:
        achieved = cmp_per_launch / (ms / 1000.0) if ms > 0 else float("nan")
        return {"bound": "alu", "achieved": achieved / 1e12, "peak": self.peak_popc / 1e12, "unit": "Tcmp/s",
                "frac": achieved / self.peak_popc, "frac_popc": achieved / self.peak_popc,
                "frac_int4": achieved / self.peak_int4, "peak_int4": self.peak_int4 / 1e12,
                "traffic": traffic, "kernel": kernel, "cmp_per_launch": cmp_per_launch,
                "verify_ms_per_launch": ms,
                "peak_basis": f"one POPC per comparison: {self.popc:.2f} POPC/clk/SM (measured probe) x {self.sms} "
                              f"SMs x {self.fmax/1e6:.0f} MHz (of measured); frac_int4 against {self.sms} SMs x "
                              f"128 lanes x {self.fmax/1e6:.0f} MHz / 4 issue slots per comparison; comparison-mix "
                              f"probe {self.mix:.2f}/clk/SM",
                "share_of_step": share}


def measure_plain(pms, torch, dev, stream, peaks, l, d, K, Wm, rank, dist, q: int = 0, clk=None) -> dict:
    """One plain configuration: K timed device-resident solves (CUDA events on the library stream,
    L2 flushed between steps; the captured graphs replay without timing events), the same K
    solves again with the device-time events inside the graphs (pms_options.graph = 1) for the
    verification kernel's own duration, its comparisons (count mode, same instances), and K
    end-to-end solves from host memory through pms_solve."""
    n, m = 20, 600
    seeds = rank_seeds(rank, K + Wm)
    insts = [pi.planted_instance(n, m, l, d, s) for s in seeds]
    d_in = [torch.from_numpy(i.seqs.copy()).to(dev) for i in insts]
    cap = 1 << 16
    d_out = torch.zeros(cap, dtype=torch.int64, device=dev)
    d_st = torch.zeros(4, dtype=torch.int32, device=dev)
    ctx = pms.Context(dev.index)
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

    # the verification kernel's duration: the same steps through graphs that carry the
    # device-time events (an event node between two kernels costs their launch overlap,
    # so the value pass runs without them)
    tctx = pms.Context(dev.index)
    tctx.set_stream(stream)
    tctx.set_options(graph=1, quorum=q)
    for i in range(Wm):
        with torch.cuda.stream(stream):
            tctx.solve_device(d_in[i], n, m, l, d, d_out, cap, d_st)
    stream.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    tev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    verify_ms = []
    barrier(dist)
    torch.cuda.synchronize(dev)
    with (clk if clk is not None else _Null()):
        for k in range(K):
            with torch.cuda.stream(stream):
                flush(k)
                ev[k][0].record(stream)
                ctx.solve_device(d_in[Wm + k], n, m, l, d, d_out, cap, d_st)
                ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        for k in range(K):
            with torch.cuda.stream(stream):
                flush(k)
                tev[k][0].record(stream)
                tctx.solve_device(d_in[Wm + k], n, m, l, d, d_out, cap, d_st)
                tev[k][1].record(stream)
            s = tctx.stats()   # waits for this step's kernels
            assert s["ms_verify"] > 0, "timed graph replay without a verification time"
            verify_ms.append(s["ms_verify"])
        torch.cuda.synchronize(dev)
    barrier(dist)
    tctx.close()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    timed_step_ms = statistics.mean(a.elapsed_time(b) for a, b in tev)
    total_ms = max_over_ranks(dist, sum(step_ms))
    solves = sum_over_ranks(dist, K)
    value = solves / (total_ms / 1000.0)

    # algorithmic work of the dominant kernel (count mode, same instances, untimed)
    cctx = pms.Context(dev.index)
    cctx.set_options(count_work=1, quorum=q)
    cmp_total = tested = 0
    for k in range(K):
        cctx.solve(insts[Wm + k].seqs, l, d)
        s = cctx.stats()
        # comparisons of the verification kernel only (the (n - 1) W^2 of the
        # compatibility masks are another kernel's)
        cmp_total += s["cmp_reduce"] + s["cmp_verify"]
        tested += s["candidates_tested"]
    cctx.close()
    verify_avg_ms = statistics.mean(verify_ms)

    # e2e through the host-buffer C-ABI call: the inputs cross from pinned host
    # memory (read there by the packing kernel) and the status block and codes
    # back (written there by the sort kernel)
    e2e_ms, e2e_codes = [], 0
    torch.cuda.synchronize(dev)
    for k in range(K):
        flush(k)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        res = ctx.solve(insts[Wm + k].seqs, l, d)
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
        e2e_codes += len(res)
    e2e_total = max_over_ranks(dist, sum(e2e_ms))
    ctx.close()
    W = m - l + 1
    tested_total = sum_over_ranks(dist, tested)
    return {
        "value": value, "unit": "solves/s", "steps": K, "warmup": Wm, "ms_per_step": total_ms / K,
        "config": {"workload": (f"quorum ({l},{d}) q={q}" if q else f"plain ({l},{d})")
                               + f" n={n} m={m}, one seeded FM-model instance per step",
                   "l": l, "d": d, "n": n, "m": m, "l2": "flushed between steps (512 MiB write, untimed)",
                   "timing": "CUDA events on the library stream around pms_solve_device; graphs replayed "
                             "without timing events (pms_options.graph = 0)"},
        # the second pass over the same steps, graphs with the device-time events inside
        "kernel_timing_pass": {"ms_per_step": timed_step_ms, "verify_ms": statistics.mean(verify_ms),
                               "graph": "pms_options.graph = 1 (event nodes around each kernel)"},
        # candidates generated and compared explicitly against occurrences (count mode)
        "candidate_checks_per_s": tested_total / (total_ms / 1000.0),
        "candidates_tested_per_step": tested / K,
        # the searched space W * |B(x, d)| per solve, for scale (not checks)
        "search_space_per_s": solves * W * (n - q + 1 if q else 1) * n_ball(l, d) / (total_ms / 1000.0),
        "roofline": peaks.roofline(cmp_total / K, verify_avg_ms, "main_kernel (verification)",
                                   measured_traffic("pms_kernels.cu", f"quorum{l}_{d}_q{q}" if q else f"plain{l}_{d}"),
                                   verify_avg_ms / timed_step_ms),
        "e2e": {"value": solves / (e2e_total / 1000.0), "unit": "solves/s", "h2d_bytes_per_step": n * m,
                "d2h_bytes_per_step": 16 + 8 * e2e_codes / K, "ms_per_step": e2e_total / K},
        "gpu_launches": 3 * K,   # packing + compatibility masks, verification, sort/unique
    }


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


def bench_plain(args, ws, rank, local, dist, l, d, q: int = 0, extras: bool = False) -> dict:
    import torch
    import paper_2403_00306_gb300 as pms
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    pctx = pms.Context(local)
    peaks = Peaks(pctx, torch, dev)
    pctx.close()
    clk = ClockSampler(local)
    r = measure_plain(pms, torch, dev, stream, peaks, l, d, args.steps, args.warmup, rank, dist, q, clk=clk)
    line = {"metric": METRIC, "value": r["value"], "unit": "solves/s", "n_gpus": ws, "steps": r["steps"],
            "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": r["config"]}
    for k in ("candidate_checks_per_s", "candidates_tested_per_step", "search_space_per_s", "roofline",
              "kernel_timing_pass", "e2e", "gpu_launches"):
        line[k] = r[k]
    line["clocks"] = clk.summary()
    if extras:
        # the other BASELINE configurations, each measured the same way (fewer steps)
        per = {}
        for (pl, pd), steps in (((9, 2), 10), ((17, 5), 5), ((19, 6), 3)):
            c2 = ClockSampler(local)
            pr = measure_plain(pms, torch, dev, stream, peaks, pl, pd, steps, 3, rank, dist, clk=c2)
            pr["clocks"] = c2.summary()
            del pr["config"]["l2"]
            per[f"plain{pl}_{pd}"] = pr
        line["per_config"] = per
        line["batch"] = measure_batch(pms, torch, dev, peaks, args, rank, dist)
        line["served"] = measure_serve(pms, torch, dev, args, rank, dist)
        line["gpu_launches"] += sum(v["gpu_launches"] for v in per.values())
    return line


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
    peaks = Peaks(ctx, torch, dev)
    flush = make_flush(torch, dev)
    for i in range(Wm):
        ctx.solve_sigma(insts[i].seqs, l, d, pi.PROTEIN)
    kern_ms, verify_ms, e2e_ms, cmps, tested, letters = [], [], [], [], [], 0
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
            tested.append(s["candidates_tested"])
            assert insts[Wm + k].motif in {bytes(r) for r in out}, "planted motif missing"
            letters += out.size
        torch.cuda.synchronize(dev)
    barrier(dist)
    total_ms = max_over_ranks(dist, sum(kern_ms))
    solves = sum_over_ranks(dist, K)
    value = solves / (total_ms / 1000.0)
    e2e_total = max_over_ranks(dist, sum(e2e_ms))
    verify_avg = statistics.mean(verify_ms)
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
        "candidate_checks_per_s": sum(tested) / (sum(kern_ms) / 1000.0),
        "search_space_per_s": solves * W * n_ball(l, d, 20) / (total_ms / 1000.0),
        "roofline": peaks.roofline(statistics.mean(cmps), verify_avg, "sigma_main_kernel (search)",
                                   measured_traffic("pms_sigma.cu", f"protein{l}_{d}"),
                                   verify_avg / (total_ms / K)),
        # up: the letters; down: the 112-byte counter block and the motifs' letters
        "e2e": {"value": solves / (e2e_total / 1000.0), "unit": "solves/s", "h2d_bytes_per_step": n * m,
                "d2h_bytes_per_step": 112 + letters / K, "ms_per_step": e2e_total / K},
        "gpu_launches": 3 * K,   # packing, search, sort/unique
        "clocks": clocks,
    }


def measure_batch(pms, torch, dev, peaks, args, rank, dist, steps: int = 3) -> dict:
    """256 mixed instances in one persistent launch (autotuned schedule) against the same
    instances solved one by one on the plain path."""
    insts = pi.batch_instances(count=256, master_seed=2024 + rank)
    ctx = pms.Context(dev.index)
    batch = [(i.seqs, i.l, i.d) for i in insts]
    t_tune = time.perf_counter()
    # tunes each (l, d, n, m) class once, untimed; graph = 1: the replays carry the
    # device-time events (about 17 us against a launch of hundreds of milliseconds)
    ctx.set_options(autotune=1, graph=1)
    ctx.solve_batch(batch)
    t_tune = time.perf_counter() - t_tune
    for _ in range(3):
        ctx.solve_batch(batch)
    flush = make_flush(torch, dev)
    barrier(dist)
    wall, kern, ver = [], [], []
    with ClockSampler(dev.index) as clk:
        for k in range(steps):
            flush(k)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            res = ctx.solve_batch(batch)
            wall.append(time.perf_counter() - t0)
            s = ctx.stats()
            kern.append(s["ms_kernel"])
            ver.append(s["ms_verify"])
    barrier(dist)
    replays = ctx.stats()["graph_replays"]
    # one by one on the plain path (pms_solve, host buffers; device time from the stats)
    one_wall, one_kern = [], []
    for k in range(max(1, steps - 1)):
        tw = tk = 0.0
        for i in insts:
            t0 = time.perf_counter()
            ctx.solve(i.seqs, i.l, i.d)
            tw += time.perf_counter() - t0
            tk += ctx.stats()["ms_kernel"]
        one_wall.append(tw)
        one_kern.append(tk)
    # verification-kernel work (count mode, untimed)
    cctx = pms.Context(dev.index)
    cctx.set_options(count_work=1)
    cctx.solve_batch(batch)
    cs = cctx.stats()
    cctx.close()
    ctx.close()
    ok = all(not isinstance(r, Exception) for r in res)
    kern_ms = statistics.mean(kern)
    ver_ms = statistics.mean(ver)
    solves = sum_over_ranks(dist, 256)
    return {"workload": "batch of 256 instances (master seed 2024), (l,d) in {(11,3),(13,4),(15,4)}, "
                        "n in [10,30], m in [300,1000]",
            "value": solves / (max_over_ranks(dist, kern_ms) / 1000.0), "unit": "solves/s",
            "timing": "value: device time of the batch pipeline (CUDA events, first to last kernel); e2e: "
                      "host clock around pms_solve_batch (upload, kernels, download)",
            "steps": steps, "ms_per_step": kern_ms,
            "e2e": {"value": solves / max_over_ranks(dist, statistics.mean(wall)), "unit": "solves/s",
                    "ms_per_step": 1000 * statistics.mean(wall),
                    "h2d_bytes_per_step": int(sum(i.n * i.m for i in insts)),
                    "d2h_bytes_per_step": int(16 * 256 + 8 * sum(len(r) for r in res if not isinstance(r, Exception)))},
            "one_by_one": {"value": 256 / (statistics.mean(one_kern) / 1000.0), "unit": "solves/s",
                           "timing": "sum of the device times of 256 pms_solve calls",
                           "e2e_value": 256 / statistics.mean(one_wall)},
            "verify_ms": ver_ms, "share_verify": ver_ms / kern_ms,
            "other_kernels_ms": kern_ms - ver_ms,   # packing, compatibility masks, sort/unique
            "graph_replays_after_timed_steps": replays,
            "candidate_checks_per_s": cs["candidates_tested"] / (kern_ms / 1000.0),
            "roofline": peaks.roofline(cs["cmp_reduce"] + cs["cmp_verify"], ver_ms, "main_kernel (verification)",
                                       None, ver_ms / kern_ms),
            "all_ok": ok, "autotune_s": t_tune, "gpu_launches": 4 * steps, "clocks": clk.summary()}


def measure_serve(pms, torch, dev, args, rank, dist, tune: bool = True) -> dict:
    """Poisson request stream through the served form (continuous batching). With `tune`, every
    instance class of the stream (l, d, n, m rounded up to a power of two) is autotuned first,
    untimed, as a service would do once for the shapes it expects."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    count, rate = args.serve_requests, args.serve_rate
    reqs = list(pi.serve_requests(count=count, rate_per_s=rate, master_seed=7 + rank))
    ctx = pms.Context(dev.index)
    t_tune = time.perf_counter()
    classes = {}
    if tune:
        for _, inst in reqs:
            key = (inst.l, inst.d, 1 << (inst.n - 1).bit_length(), 1 << (inst.m - 1).bit_length())
            classes.setdefault(key, inst)
        for inst in classes.values():
            ctx.autotune(inst.n, inst.m, inst.l, inst.d)
    t_tune = time.perf_counter() - t_tune
    for _, inst in reqs[:8]:      # warm-up, not timed
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
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        futs = []
        for i, (ta, inst) in enumerate(reqs):
            target = t0 + ta
            delay = target - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            arrival = target
            t = ctx.submit(inst.seqs, inst.l, inst.d)
            futs.append(pool.submit(waiter, i, t, arrival))
        for f in futs:
            f.result()
        t_end = max(done_t)
    pool.shutdown()
    st = ctx.stats()
    # saturation: a slice of the stream submitted at once
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
    return {"workload": f"served: {count} Poisson requests at {rate:g}/s (master seed 7), (l,d) in "
                        "{(13,4),(15,4),(17,5)}, n=20, m in [200,1200]",
            "value": solves / span_max, "unit": "solves/s", "requests": count,
            "timing": "host clock from each request's arrival time to pms_wait's return; value = requests / "
                      "(last completion - first arrival)",
            "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[int(len(lat_ms) * 0.99) - 1],
                           "max": lat_ms[-1]},
            "offered_per_s": rate, "saturation_solves_per_s": sat, "saturation_requests": sat_n,
            "all_ok": all(ok), "tuned_classes": len(classes), "autotune_s": t_tune,
            "serve": {"waves": st["serve_waves"], "overlapped_waves": st["serve_overlapped_waves"],
                      "max_requests_per_wave": st["serve_max_requests_per_wave"]},
            "e2e": {"value": solves / span_max, "unit": "solves/s",
                    "h2d_bytes_per_step": int(statistics.mean(i.n * i.m for _, i in reqs)),
                    "d2h_bytes_per_step": 16 + 512 * 8},
            "gpu_launches": 3 * count + int(st["serve_waves"]), "clocks": clk.summary()}


def bench_onehot(args, ws, rank, local, dist) -> dict:
    """The one-hot tensor-core form of the candidate-versus-window distance, timed as a library GEMM.

    With every l-mer as a one-hot vector of 4l entries (padded to 64), the number of positions
    where a candidate c and a window w agree is the dot product of their vectors, so all
    candidate-by-window distances of a seed are one GEMM: (|B(x, d)| x 64) by (64 x windows of
    the other n - 1 sequences). This times that GEMM (torch.matmul, bf16, cuBLAS: a timing copy,
    not part of the library) for one (15,4) seed, n = 20, m = 600, on one-hot inputs built from
    a seeded instance, and scales it by the seeds of a solve. The tree search of the library
    needs no such contraction; this line measures what the dense form would cost."""
    import torch
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    l, d, n, m = 15, 4, 20, 600
    inst = pi.plain_instance(l, d, seed=1)
    codes = np.frombuffer(b"ACGT", dtype=np.uint8)
    lut = np.zeros(256, dtype=np.int64)
    lut[codes] = np.arange(4)
    seq = lut[inst.seqs]                              # n x m letter indices
    W = m - l + 1
    win = np.stack([seq[:, j:j + l] for j in range(W)], axis=1)[1:].reshape(-1, l)   # (n-1)W x l
    K = 64
    Wt = np.zeros((win.shape[0], K), dtype=np.float32)
    Wt[np.arange(win.shape[0])[:, None], 4 * np.arange(l)[None, :] + win] = 1.0
    # the candidates of one seed: B(x, d) enumerated position set by position set
    x = seq[0, :l]
    cand = [x.copy()]
    import itertools
    for k in range(1, d + 1):
        for P in itertools.combinations(range(l), k):
            for lets in itertools.product(range(3), repeat=k):
                c = x.copy()
                for p, t in zip(P, lets):
                    c[p] = (x[p] + 1 + t) % 4
                cand.append(c)
    cand = np.array(cand)
    C = np.zeros((len(cand), K), dtype=np.float32)
    C[np.arange(len(cand))[:, None], 4 * np.arange(l)[None, :] + cand] = 1.0
    A = torch.from_numpy(C).to(dev, torch.bfloat16)
    B = torch.from_numpy(Wt.T.copy()).to(dev, torch.bfloat16)
    out = torch.empty(A.shape[0], B.shape[1], device=dev, dtype=torch.bfloat16)
    for _ in range(3):
        torch.matmul(A, B, out=out)
    torch.cuda.synchronize(dev)
    # agreement: matches >= l - d somewhere in each sequence (checked once, untimed)
    hits = (out.float() >= l - d).view(len(cand), n - 1, W).any(dim=2).all(dim=1)
    reps = max(3, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record()
        for _ in range(reps):
            torch.matmul(A, B, out=out)
        e1.record()
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * A.shape[0] * K * B.shape[1]
    peaks = load_peaks()
    solve_ms = ms * W
    return {"metric": METRIC, "value": 1000.0 / solve_ms, "unit": "solves/s", "n_gpus": ws, "steps": reps,
            "warmup": 3, "ms_per_step": solve_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "one-hot tensor-core form, plain (15,4) n=20 m=600: the GEMM of one seed's "
                                   f"{A.shape[0]} candidates by the {B.shape[1]} windows of the other sequences "
                                   "(K = 64), scaled by the 586 seeds of a solve",
                       "timing": "CUDA events around torch.matmul (cuBLAS bf16), a timing copy"},
            "gemm_ms_per_seed": ms, "gemm_tflops": flops / (ms / 1000.0) / 1e12,
            "roofline": {"bound": "tensor", "achieved": flops / (ms / 1000.0) / 1e12,
                         "peak": float(peaks.get("bf16_tflops", 1900.0)), "unit": "TFLOP/s",
                         "frac": flops / (ms / 1000.0) / 1e12 / float(peaks.get("bf16_tflops", 1900.0)),
                         "traffic": None, "kernel": "cuBLAS bf16 GEMM (timing copy)"},
            "candidates_of_seed_passing_all": int(hits.sum().item()),
            "e2e": None, "gpu_launches": reps, "clocks": clk.summary()}


def bench_batch(args, ws, rank, local, dist) -> dict:
    import torch
    import paper_2403_00306_gb300 as pms
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = pms.Context(local)
    peaks = Peaks(ctx, torch, dev)
    ctx.close()
    b = measure_batch(pms, torch, dev, peaks, args, rank, dist, steps=args.steps)
    line = {"metric": METRIC, "value": b["value"], "unit": "solves/s", "n_gpus": ws, "steps": b["steps"],
            "warmup": 3, "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": b["workload"], "timing": b["timing"], "l2": "flushed between steps"}}
    line.update({k: v for k, v in b.items() if k not in line and k not in ("workload", "timing")})
    return line


def bench_serve(args, ws, rank, local, dist) -> dict:
    import torch
    import paper_2403_00306_gb300 as pms
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    s = measure_serve(pms, torch, dev, args, rank, dist)
    line = {"metric": METRIC, "value": s["value"], "unit": "solves/s", "n_gpus": ws, "steps": s["requests"],
            "warmup": 8, "ms_per_step": 1000.0 / s["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": s["workload"], "timing": s["timing"]}}
    line.update({k: v for k, v in s.items() if k not in line and k not in ("workload", "timing", "requests")})
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="suite",
                    choices=["suite"] + sorted(WORKLOADS) + sorted(QUORUM_WORKLOADS) + sorted(PROTEIN_WORKLOADS)
                    + ["batch", "serve", "onehot15_4"],
                    help="suite (default): the plain (15,4) line, with per_config lines for (9,2), (17,5), "
                         "(19,6), the batched and the served workloads inside it")
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
    cpu = rank == 0 and ws == 1 and not args.no_cpu_baseline
    if args.workload == "onehot15_4":
        line = bench_onehot(args, ws, rank, local, dist)
    elif args.workload == "batch":
        line = bench_batch(args, ws, rank, local, dist)
    elif args.workload == "serve":
        line = bench_serve(args, ws, rank, local, dist)
    elif args.workload in PROTEIN_WORKLOADS:
        l, d = PROTEIN_WORKLOADS[args.workload]
        line = bench_sigma(args, ws, rank, local, dist, l, d)
        if cpu:
            c = cpu_oracle_slice(l, d, 20, 600, 424242, 15.0, os.cpu_count() or 1, alphabet=pi.PROTEIN)
            line["cpu_baseline"] = {"value": c["value"], "unit": "solves/s", "cores": os.cpu_count() or 1,
                                    "kind": "oracle", "threads": c["threads"], "sample": c["sample"]}
    else:
        suite = args.workload == "suite"
        l, d, q = QUORUM_WORKLOADS[args.workload] if args.workload in QUORUM_WORKLOADS \
            else (*WORKLOADS["plain15_4" if suite else args.workload], 0)
        line = bench_plain(args, ws, rank, local, dist, l, d, q, extras=suite)
        if cpu:
            if q:
                c = cpu_oracle_slice(l, d, 20, 600, 424242, 15.0, os.cpu_count() or 1, q=q)
                line["cpu_baseline"] = {"value": c["value"], "unit": "solves/s", "cores": os.cpu_count() or 1,
                                        "kind": "oracle", "threads": c["threads"], "sample": c["sample"]}
            else:
                line["cpu_baseline"] = cpu_baseline_plain(l, d)
            if suite:
                for name, pc in line["per_config"].items():
                    pl, pd = WORKLOADS[name]
                    pc["cpu_baseline"] = cpu_baseline_plain(pl, pd)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
