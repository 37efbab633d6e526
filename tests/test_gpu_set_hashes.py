"""GPU motif sets against oracle-written sizes and hashes of whole motif sets.

golden/set_hashes.json holds, for every one of the 256 instances of the batched workload
and for a random sample of the served stream's requests (a prefix of a random order of
requests 16..9999, at least 32), the size of the oracle's whole motif set and a SHA-256 of
its sorted codes (written by golden/make_set_hashes.py, which calls only the oracle). The
GPU's sorted codes are hashed the same way, so each comparison is bit-exact.
"""
import hashlib
import importlib.util
import json
import os

import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GOLD = json.load(open(os.path.join(GOLDEN, "set_hashes.json")))
BATCH = sorted((g for g in GOLD.values() if g["kind"] == "batch"), key=lambda g: g["index"])
SERVED = sorted((g for g in GOLD.values() if g["kind"] == "serve"), key=lambda g: g["rank"])


def _served_order():
    spec = importlib.util.spec_from_file_location("make_set_hashes", os.path.join(GOLDEN, "make_set_hashes.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.served_order()


def _seq_hash(seqs):
    return hashlib.sha256(np.ascontiguousarray(seqs, dtype=np.uint8).tobytes()).hexdigest()[:16]


def _set_hash(codes):
    return hashlib.sha256(np.asarray(codes, dtype="<u8").tobytes()).hexdigest()


def _check(g, inst, got):
    assert _seq_hash(inst.seqs) == g["seq_sha256_16"], "the instance generator changed since the hashes were written"
    assert (inst.n, inst.m, inst.l, inst.d) == (g["n"], g["m"], g["l"], g["d"])
    assert len(got) == g["count"], (g["kind"], g["index"], len(got), g["count"])
    assert _set_hash(got) == g["motifs_sha256"], (g["kind"], g["index"])


def test_the_hash_file_is_complete():
    assert [g["index"] for g in BATCH] == list(range(256))
    # the served entries are a prefix of the sampling order: a random sample, not a chosen one
    assert len(SERVED) >= 32
    assert [g["rank"] for g in SERVED] == list(range(len(SERVED)))
    assert [g["index"] for g in SERVED] == _served_order()[:len(SERVED)]


def test_all_256_batched_instances_against_the_oracle():
    insts = pi.batch_instances(count=256, master_seed=2024)
    c = pms.Context(0)
    # three calls: kernel by kernel, captured as a graph, replayed
    for call in range(3):
        res = c.solve_batch([(i.seqs, i.l, i.d) for i in insts])
        for g, inst, r in zip(BATCH, insts, res):
            assert not isinstance(r, Exception), (call, g["index"], r)
            _check(g, inst, r)
    assert c.stats()["graph_replays"] >= 1
    c.close()


def test_served_random_requests_against_the_oracle():
    reqs = list(pi.serve_requests(count=10000, master_seed=7))
    sample = [reqs[g["index"]][1] for g in SERVED]
    c = pms.Context(0)
    tickets = [c.submit(r.seqs, r.l, r.d) for r in sample]   # all in flight together
    for g, r, t in zip(SERVED, sample, tickets):
        got = c.wait(t, 300000)
        _check(g, r, got)
        c.release(t)
    c.close()
