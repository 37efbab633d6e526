#!/usr/bin/env python3
"""Writes set_hashes.json: the size and a SHA-256 of the whole motif set of each instance below,
computed by the CPU oracle only (``oracle.Oracle.solve_packed``: Definitions 3-5 with q = n,
candidates from B(x, d) over the l-mers x of s_1, Observation 3.1; pinned against the char-level
solver and brute force in oracle_pins.check_packed_solver). Nothing from the GPU library is
imported. A hash stands in for the set itself because some sets are large (up to about 400,000
codes); the test hashes the GPU's sorted codes the same way, so the comparison stays bit-exact.

Hash: SHA-256 of the sorted unique motif codes (2 bits per base, position 0 most significant)
as little-endian 64-bit words.

Entries:
  batch2024_{0..255}  every instance of the batched workload (master seed 2024)
  serve7_r{k}         requests of the served stream (master seed 7, 10,000 requests,
                      m in [200, 1200]) in a uniformly random order of requests 16..9999
                      (requests 0..15 are checked whole in whole_sets.json): first 32 drawn
                      with generator seed 7007, then the others in a random permutation
                      (generator seed 7008). The file holds a prefix of that order; a longer
                      run extends it (--serve N: the first N of the order).

Usage: python tests/golden/make_set_hashes.py [--serve N] [--threads T] [name-prefix ...]
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

OUT = os.path.join(HERE, "set_hashes.json")
SERVE_SAMPLE = 32
SERVE_SAMPLE_SEED = 7007


def seq_hash(seqs: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(seqs, dtype=np.uint8).tobytes()).hexdigest()[:16]


def set_hash(codes) -> str:
    return hashlib.sha256(np.asarray(codes, dtype="<u8").tobytes()).hexdigest()


def served_order() -> list[int]:
    """Requests 16..9999 in the order the served sample takes them."""
    rng = np.random.default_rng(SERVE_SAMPLE_SEED)
    first = sorted(int(k) for k in rng.choice(np.arange(16, 10000), size=SERVE_SAMPLE, replace=False))
    taken = set(first)
    rest = np.array([k for k in range(16, 10000) if k not in taken])
    return first + [int(k) for k in np.random.default_rng(SERVE_SAMPLE_SEED + 1).permutation(rest)]


def entries(serve: int):
    for k, inst in enumerate(pi.batch_instances(count=256, master_seed=2024)):
        yield f"batch2024_{k}", {"kind": "batch", "index": k, "master_seed": 2024}, inst
    reqs = list(pi.serve_requests(count=10000, master_seed=7))
    for rank, k in enumerate(served_order()[:serve]):
        yield f"serve7_r{k}", {"kind": "serve", "index": k, "rank": rank, "master_seed": 7}, reqs[k][1]


def main(argv):
    args = argv[1:]
    serve, threads = SERVE_SAMPLE, os.cpu_count() or 1
    while args and args[0] in ("--serve", "--threads"):
        if args[0] == "--serve":
            serve = int(args[1])
        else:
            threads = int(args[1])
        args = args[2:]
    redo = args
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    o = oracle.Oracle()
    for name, desc, inst in entries(serve):
        if name in data and not any(name.startswith(p) for p in redo):
            if "rank" in desc and data[name].get("rank") != desc["rank"]:
                data[name]["rank"] = desc["rank"]   # entries written before ranks were recorded
            continue
        t0 = time.perf_counter()
        codes = o.solve_packed(inst.seqs, inst.l, inst.d, threads=threads, cap=1 << 24)
        assert np.all(np.diff(codes.astype(np.uint64)) > 0) or len(codes) <= 1
        data[name] = dict(desc, n=inst.n, m=inst.m, l=inst.l, d=inst.d, seq_sha256_16=seq_hash(inst.seqs),
                          count=int(len(codes)), motifs_sha256=set_hash(codes),
                          oracle_s=round(time.perf_counter() - t0, 1))
        tmp = OUT + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=0, sort_keys=True)
        os.replace(tmp, OUT)
        print(f"{name}: {len(codes)} motifs in {data[name]['oracle_s']} s", flush=True)


if __name__ == "__main__":
    main(sys.argv)
