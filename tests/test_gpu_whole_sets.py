"""GPU motif sets of full-size instances against whole motif sets written by the CPU oracle.

The expected sets are in golden/whole_sets.json, written by
golden/make_whole_sets.py, which calls only the oracle (Definitions 3-5 with
q = n; the answer is a set of strings, so the comparison is bit-exact).
Covered: plain (15,4) seeds 1-3 and (17,5) seed 1 whole; (19,6) seed 1 on 48
seeds of s_1 (the last 24 windows, whose items the work queue's tail split
cuts into chunks, the planted copy's window and 23 random ones); the first 32
instances of the batched workload through one batched launch (default and
autotuned schedules); the first 16 requests of the served stream (m up to
1200, rows beyond shared memory included) submitted together.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms
from parity_helpers import keys_within, py_key, seq_codes

pytestmark = pytest.mark.gpu

GOLD_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "whole_sets.json")
GOLD = json.load(open(GOLD_PATH))


def _checked(name, inst):
    g = GOLD[name]
    h = hashlib.sha256(np.ascontiguousarray(inst.seqs, dtype=np.uint8).tobytes()).hexdigest()[:16]
    assert h == g["seq_sha256_16"], f"{name}: the instance generator changed since the expected set was written"
    assert (inst.n, inst.m, inst.l, inst.d) == (g["n"], g["m"], g["l"], g["d"])
    return g


def _want(name, inst):
    return np.array(_checked(name, inst)["motifs"], dtype=np.uint64)


@pytest.fixture(scope="module")
def ctx():
    c = pms.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["plain15_4_s1", "plain15_4_s2", "plain15_4_s3", "plain17_5_s1"])
def test_plain_whole_motif_set(ctx, name):
    import torch
    g = GOLD[name]
    inst = pi.plain_instance(g["l"], g["d"], seed=g["seed"])
    want = _want(name, inst)
    assert py_key(inst.motif.decode()) in set(int(k) for k in want)
    assert np.array_equal(ctx.solve(inst.seqs, inst.l, inst.d), want)
    # the launch configuration the benchmark times: device buffers on a side
    # stream, the plan captured as a graph on its second call and replayed after
    stream = torch.cuda.Stream()
    c = pms.Context(0)
    c.set_stream(stream)
    d_in = torch.from_numpy(inst.seqs.copy()).cuda()
    cap = 1 << 16
    for _ in range(3):
        out = torch.zeros(cap, dtype=torch.int64, device="cuda")
        st = torch.zeros(4, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            c.solve_device(d_in, inst.n, inst.m, inst.l, inst.d, out, cap, st)
        stream.synchronize()
        s = st.cpu().numpy().astype(np.uint32)
        assert s[2] == 0
        assert np.array_equal(out[: int(s[1])].cpu().numpy().astype(np.uint64), want)
    c.close()


@pytest.mark.parametrize("smem_rows", [256, 128])
def test_plain_whole_motif_set_rows_off_chip(smem_rows):
    # (15,4) seeds hold about 630 feasible occurrences: with 256 entries of shared memory the
    # mismatch masks stay there and the planes are read from global memory; with 128 both are
    # read from global memory
    for name in ("plain15_4_s1", "plain15_4_s2"):
        g = GOLD[name]
        inst = pi.plain_instance(g["l"], g["d"], seed=g["seed"])
        c = pms.Context(0)
        c.set_options(smem_rows=smem_rows)
        assert np.array_equal(c.solve(inst.seqs, inst.l, inst.d), _want(name, inst)), (name, smem_rows)
        c.close()


def test_plain_19_6_on_48_seeds(ctx):
    g = GOLD["plain19_6_s1"]
    inst = pi.plain_instance(19, 6, seed=1)
    _checked("plain19_6_s1", inst)
    got = ctx.solve(inst.seqs, 19, 6)
    assert np.all(np.diff(got.astype(np.int64)) > 0) or len(got) <= 1
    codes = seq_codes(inst.seqs[0])
    assert len(g["per_seed"]) == 48
    for j, keys in g["per_seed"].items():
        j = int(j)
        mine = keys_within(got, codes[j:j + 19], 19, 6)
        assert np.array_equal(mine, np.array(keys, dtype=np.uint64)), (j, len(mine), len(keys))
    assert py_key(inst.motif.decode()) in set(int(k) for k in got)


@pytest.mark.parametrize("name,triple_rows", [("plain15_4_s1", 4), ("plain15_4_s2", 19), ("plain17_5_s1", 8),
                                              ("plain17_5_s1", 19)])
def test_plain_whole_motif_set_three_string(name, triple_rows):
    g = GOLD[name]
    inst = pi.plain_instance(g["l"], g["d"], seed=g["seed"])
    c = pms.Context(0)
    c.set_options(triple_rows=triple_rows)
    assert np.array_equal(c.solve(inst.seqs, inst.l, inst.d), _want(name, inst))
    c.close()


def test_plain_19_6_on_48_seeds_three_string():
    g = GOLD["plain19_6_s1"]
    inst = pi.plain_instance(19, 6, seed=1)
    _checked("plain19_6_s1", inst)
    c = pms.Context(0)
    c.set_options(triple_rows=8)
    got = c.solve(inst.seqs, 19, 6)
    c.close()
    codes = seq_codes(inst.seqs[0])
    for j, keys in g["per_seed"].items():
        j = int(j)
        assert np.array_equal(keys_within(got, codes[j:j + 19], 19, 6), np.array(keys, dtype=np.uint64)), j


def _batch_slice():
    insts = pi.batch_instances(count=256, master_seed=2024)[:32]
    return insts, [_want(f"batch2024_{k}", inst) for k, inst in enumerate(insts)]


@pytest.mark.parametrize("autotune", [0, 1])
def test_batch_slice_whole_motif_sets(autotune):
    insts, wants = _batch_slice()
    c = pms.Context(0)
    if autotune:
        c.set_options(autotune=1)
    # three calls: kernel by kernel, captured as a graph, replayed
    for call in range(3):
        res = c.solve_batch([(i.seqs, i.l, i.d) for i in insts])
        for k, (r, want) in enumerate(zip(res, wants)):
            assert not isinstance(r, Exception), (call, k, r)
            assert np.array_equal(r, want), (call, k, insts[k].l, insts[k].d, insts[k].n, insts[k].m, len(r), len(want))
    c.close()


def test_served_requests_whole_motif_sets():
    reqs = [inst for _, inst in pi.serve_requests(count=16, master_seed=7)]
    wants = [_want(f"serve7_{k}", inst) for k, inst in enumerate(reqs)]
    assert max(r.m for r in reqs) >= 1100
    c = pms.Context(0)
    tickets = [c.submit(r.seqs, r.l, r.d) for r in reqs]    # all arrive while the first ones run
    for k, (t, want) in enumerate(zip(tickets, wants)):
        got = c.wait(t, 120000)
        assert np.array_equal(got, want), (k, reqs[k].l, reqs[k].d, reqs[k].m, len(got), len(want))
        c.release(t)
    s = c.stats()
    assert s["serve_overlapped_waves"] >= 1 and s["serve_max_requests_per_wave"] >= 2
    c.close()
