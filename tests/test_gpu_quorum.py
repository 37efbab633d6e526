"""Quorum form (qPMS, q < n) against the oracle's quorum solver, bit-exact."""
import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms
from parity_helpers import keys_within, oracle_per_seed, py_key, seq_codes

pytestmark = pytest.mark.gpu

SMALL_Q = [
    # (n, m, l, d, seed, q)
    (2, 30, 6, 2, 2, 1),
    (3, 8, 8, 2, 3, 2),
    (4, 40, 5, 1, 4, 2),
    (5, 50, 6, 0, 5, 3),
    (6, 60, 6, 2, 6, 4),
    (8, 100, 9, 2, 8, 5),
    (8, 100, 9, 2, 8, 7),
    (10, 200, 11, 3, 9, 8),
    (12, 64, 7, 1, 15, 6),
    (7, 90, 10, 3, 21, 5),
]


def _ctx(q, **kw):
    c = pms.Context(0)
    c.set_options(quorum=q, **kw)
    return c


@pytest.mark.parametrize("case", SMALL_Q, ids=lambda c: "n{}_m{}_l{}_d{}_q{}".format(c[0], c[1], c[2], c[3], c[5]))
def test_quorum_small_match_oracle(oracle_, case):
    n, m, l, d, seed, q = case
    c = _ctx(q)
    inst = pi.planted_instance(n, m, l, d, seed)
    want = oracle_.solve_quorum(inst.seqs, l, d, q, cap=1 << 24)
    got = c.solve(inst.seqs, l, d)
    assert np.array_equal(got, want), (len(got), len(want))
    seqs = pi.random_sequences(n, m, seed + 999)
    assert np.array_equal(c.solve(seqs, l, d), oracle_.solve_quorum(seqs, l, d, q, cap=1 << 24))
    c.close()


def test_quorum_rows_in_global_scratch(oracle_):
    for (n, m, l, d, seed, q) in SMALL_Q[:6]:
        c = _ctx(q, smem_rows=8)
        inst = pi.planted_instance(n, m, l, d, seed)
        assert np.array_equal(c.solve(inst.seqs, l, d), oracle_.solve_quorum(inst.seqs, l, d, q, cap=1 << 24))
        c.close()


def test_quorum_n_equals_pms():
    inst = pi.plain_instance(13, 4, seed=5)
    a = _ctx(20)
    b = pms.Context(0)
    assert np.array_equal(a.solve(inst.seqs, 13, 4), b.solve(inst.seqs, 13, 4))
    a.close()
    b.close()


def _sampled(oracle_, l, d, q, seed, seeds_per_seq, seqs_used):
    inst = pi.plain_instance(l, d, seed=seed)
    c = _ctx(q)
    got = c.solve(inst.seqs, l, d)
    c.close()
    assert py_key(inst.motif.decode()) in set(int(k) for k in got)
    W = inst.m - l + 1
    rng = np.random.default_rng(seed)
    seeds = []
    for si in seqs_used:
        seeds += [si * W + int(j) for j in rng.choice(W, size=seeds_per_seq, replace=False)]
    codes = seq_codes(inst.seqs)
    import os
    from concurrent.futures import ThreadPoolExecutor

    def one(g):
        return g, oracle_.solve_quorum_seeds(inst.seqs, l, d, q, g, g + 1, threads=1, cap=1 << 24)

    with ThreadPoolExecutor(os.cpu_count() or 2) as ex:
        want = dict(ex.map(one, seeds))
    for g, w in want.items():
        si, j = divmod(g, W)
        mine = keys_within(got, codes[si, j:j + l], l, d)
        assert np.array_equal(mine, w), (g, len(mine), len(w))


def test_quorum_full_size_11_3_q10(oracle_):
    _sampled(oracle_, 11, 3, 10, 1, 3, (0, 5, 10))


def test_quorum_full_size_15_4_q18(oracle_):
    _sampled(oracle_, 15, 4, 18, 2, 4, (0, 1, 2))
