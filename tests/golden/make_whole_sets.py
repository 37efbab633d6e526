#!/usr/bin/env python3
"""Writes whole_sets.json: expected motif sets of full-size instances, computed by the CPU oracle only.

Every set here comes from ``oracle.Oracle.solve_packed`` (Definitions 3-5 with
q = n; candidates from B(x, d) over the l-mers x of s_1, Observation 3.1; the
motif test on compressed l-mers, pinned against the char-level solver and
brute force in oracle_pins.check_packed_solver). Nothing from the GPU library
is imported. Instances are regenerated from ``planted_inputs``; each entry
stores a hash of the sequence bytes so a test can tell if the generator
changed.

Entries:
  plain15_4_s{1,2,3}  (15,4), n = 20, m = 600, seeds 1-3: whole motif sets
  plain17_5_s1        (17,5), n = 20, m = 600, seed 1: whole motif set
  plain19_6_s1        (19,6), n = 20, m = 600, seed 1: the motifs inside
                      B(x_j, 6) for 48 seeds j of s_1 (the planted copy's
                      window, the last 24 windows, 23 drawn at random)
  batch2024_{0..31}   the first 32 instances of the batched workload
                      (master seed 2024): whole motif sets
  serve7_{0..15}      the first 16 requests of the served stream (master
                      seed 7, m in [200, 1200]): whole motif sets

Usage: python tests/golden/make_whole_sets.py [name-prefix ...]
(entries already in the file are kept unless their prefix is named).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import planted_inputs as pi  # noqa: E402

OUT = os.path.join(HERE, "whole_sets.json")
SAMPLED_19_6 = 48


def seq_hash(seqs: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(seqs, dtype=np.uint8).tobytes()).hexdigest()[:16]


def sampled_seeds_19_6(inst) -> list[int]:
    W = inst.m - inst.l + 1
    seeds = {int(inst.positions[0])}
    seeds |= set(range(W - 24, W))
    rng = np.random.default_rng(19006)
    rest = [j for j in range(W) if j not in seeds]
    seeds |= set(int(j) for j in rng.choice(rest, size=SAMPLED_19_6 - len(seeds), replace=False))
    return sorted(seeds)


def entries():
    """(name, description dict, instance, seeds or None for the whole set)."""
    for s in (1, 2, 3):
        yield f"plain15_4_s{s}", {"kind": "plain", "l": 15, "d": 4, "seed": s}, pi.plain_instance(15, 4, seed=s), None
    yield "plain17_5_s1", {"kind": "plain", "l": 17, "d": 5, "seed": 1}, pi.plain_instance(17, 5, seed=1), None
    inst = pi.plain_instance(19, 6, seed=1)
    yield "plain19_6_s1", {"kind": "plain", "l": 19, "d": 6, "seed": 1}, inst, sampled_seeds_19_6(inst)
    for k, inst in enumerate(pi.batch_instances(count=256, master_seed=2024)[:32]):
        yield f"batch2024_{k}", {"kind": "batch", "index": k, "master_seed": 2024}, inst, None
    for k, (_, inst) in enumerate(pi.serve_requests(count=16, master_seed=7)):
        yield f"serve7_{k}", {"kind": "serve", "index": k, "master_seed": 7}, inst, None


def main(argv):
    redo = argv[1:]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    o = oracle.Oracle()
    threads = os.cpu_count() or 1
    for name, desc, inst, seeds in entries():
        if name in data and not any(name.startswith(p) for p in redo):
            continue
        t0 = time.perf_counter()
        rec = dict(desc, n=inst.n, m=inst.m, l=inst.l, d=inst.d, seq_sha256_16=seq_hash(inst.seqs))
        if seeds is None:
            rec["motifs"] = [int(k) for k in o.solve_packed(inst.seqs, inst.l, inst.d, threads=threads)]
        else:
            # one seed per worker thread (the library call releases the interpreter lock)
            from concurrent.futures import ThreadPoolExecutor

            def one(j):
                return str(j), [int(k) for k in o.solve_packed(inst.seqs, inst.l, inst.d, j, j + 1, threads=1)]
            with ThreadPoolExecutor(threads) as ex:
                rec["per_seed"] = dict(ex.map(one, seeds))
        rec["oracle_s"] = round(time.perf_counter() - t0, 1)
        data[name] = rec
        tmp = OUT + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=0, sort_keys=True)
        os.replace(tmp, OUT)
        print(f"{name}: {len(rec.get('motifs', rec.get('per_seed', {})))} in {rec['oracle_s']} s", flush=True)


if __name__ == "__main__":
    main(sys.argv)
