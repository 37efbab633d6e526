"""Pair seeds (Observation 3.3: candidates in B(x, d) & B(r, d) for x of s_1, r of s_2) give the
same motif sets as the oracle and as the tree form over B(x, d)."""
import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms
from parity_helpers import py_key
from test_gpu_parity import SMALL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pctx():
    c = pms.Context(0)
    c.set_options(seed_mode=1)
    yield c
    c.close()


@pytest.fixture(scope="module")
def tctx():
    c = pms.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("case", SMALL, ids=lambda c: "n{}_m{}_l{}_d{}".format(*c[:4]))
def test_pairs_small_match_oracle(pctx, oracle_, case):
    n, m, l, d, seed = case
    inst = pi.planted_instance(n, m, l, d, seed)
    assert np.array_equal(pctx.solve(inst.seqs, l, d), oracle_.solve(inst.seqs, l, d, cap=1 << 24))
    seqs = pi.random_sequences(n, m, seed + 777)
    assert np.array_equal(pctx.solve(seqs, l, d), oracle_.solve(seqs, l, d, cap=1 << 24))


@pytest.mark.parametrize("l,d,seeds", [(9, 2, (1, 2)), (11, 3, (1,)), (13, 4, (1, 2)), (15, 4, (1, 2, 3)),
                                       (17, 5, (1, 2)), (19, 6, (1,))])
def test_pairs_full_size_equal_tree(pctx, tctx, l, d, seeds):
    for seed in seeds:
        inst = pi.plain_instance(l, d, seed=seed)
        got = pctx.solve(inst.seqs, l, d)
        assert np.array_equal(got, tctx.solve(inst.seqs, l, d))
        assert py_key(inst.motif.decode()) in set(int(k) for k in got)


def test_pairs_9_2_full_size_match_oracle(pctx, oracle_):
    inst = pi.plain_instance(9, 2, seed=4)
    assert np.array_equal(pctx.solve(inst.seqs, 9, 2), oracle_.solve(inst.seqs, 9, 2))


def test_pairs_global_rows_and_batch(oracle_):
    c = pms.Context(0)
    c.set_options(seed_mode=1, smem_rows=8)
    for case in SMALL[:8]:
        n, m, l, d, seed = case
        inst = pi.planted_instance(n, m, l, d, seed)
        assert np.array_equal(c.solve(inst.seqs, l, d), oracle_.solve(inst.seqs, l, d, cap=1 << 24))
    c.close()
    c = pms.Context(0)
    c.set_options(seed_mode=1)
    base = pms.Context(0)
    insts = pi.batch_instances(count=16, master_seed=77)
    res = c.solve_batch([(i.seqs, i.l, i.d) for i in insts])
    for i, r in zip(insts, res):
        assert np.array_equal(r, base.solve(i.seqs, i.l, i.d))
    c.close()
    base.close()


def test_pairs_count_mode(pctx):
    c = pms.Context(0)
    c.set_options(seed_mode=1, count_work=1)
    inst = pi.plain_instance(15, 4, seed=2)
    got = c.solve(inst.seqs, 15, 4)
    s = c.stats()
    assert np.array_equal(got, pctx.solve(inst.seqs, 15, 4))
    assert s["candidates_tested"] > 0 and s["subsets"] > 0
    c.close()
