"""GPU motif sets against the CPU oracle, bit-exact (the answer is a set of strings: no tolerance).

Small instances are compared whole; the full-size plain configurations
(n = 20, m = 600) are compared seed by seed on sampled seeds of s_1 (the GPU
motifs inside B(x_j, d) against the oracle restricted to that seed), every
GPU motif is re-checked with the oracle's motif test, and the planted motif
must be present. All calls go through the C ABI with default options, the
launch configuration the benchmark times.
"""
import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms
from parity_helpers import keys_within, oracle_per_seed, py_key, seq_codes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pms.Context(0)
    yield c
    c.close()


SMALL = [
    # (n, m, l, d, seed) -- edge cases first
    (1, 12, 5, 1, 1),      # n = 1: every string within d of some l-mer of s_1
    (2, 30, 6, 2, 2),      # a single verified row
    (3, 8, 8, 2, 3),       # m = l: one window per sequence
    (4, 40, 1, 0, 4),      # l = 1
    (5, 50, 6, 0, 5),      # d = 0: intersection of l-mer sets
    (6, 60, 6, 3, 6),      # 2d = l: every window is a feasible occurrence
    (4, 45, 7, 4, 7),      # 2d > l
    (8, 100, 9, 2, 8),
    (10, 200, 11, 3, 9),
    (20, 120, 10, 3, 10),
    (7, 333, 12, 3, 11),   # ragged m
    (64, 50, 8, 2, 12),    # maximum n
    (3, 70, 32, 2, 13),    # maximum l
    (5, 40, 12, 5, 14),    # deep tree (d = 5) on small input
    (12, 64, 7, 1, 15),
]


@pytest.mark.parametrize("case", SMALL, ids=lambda c: "n{}_m{}_l{}_d{}".format(*c[:4]))
def test_small_instances_match_oracle(ctx, oracle_, case):
    n, m, l, d, seed = case
    inst = pi.planted_instance(n, m, l, d, seed)
    want = oracle_.solve(inst.seqs, l, d, cap=1 << 24)
    got = ctx.solve(inst.seqs, l, d)
    assert got.dtype == np.uint64
    assert np.array_equal(got, want), (len(got), len(want))
    # random, unplanted sequences of the same shape
    seqs = pi.random_sequences(n, m, seed + 777)
    assert np.array_equal(ctx.solve(seqs, l, d), oracle_.solve(seqs, l, d, cap=1 << 24))


@pytest.mark.parametrize("case", [c for c in SMALL if c[0] > 1][:10] + [(9, 301, 9, 2, 31), (16, 201, 11, 3, 32)],
                         ids=lambda c: "n{}_m{}_l{}_d{}".format(*c[:4]))
def test_rows_in_global_scratch_match_oracle(oracle_, case):
    # shared memory limited to 8 row entries: every seed's rows go to the per-CTA global scratch
    n, m, l, d, seed = case
    c = pms.Context(0)
    c.set_options(smem_rows=8)
    inst = pi.planted_instance(n, m, l, d, seed)
    assert np.array_equal(c.solve(inst.seqs, l, d), oracle_.solve(inst.seqs, l, d, cap=1 << 24))
    c.close()


DEEP = [
    # (n, m, l, d, seed) -- trees with nodes of 4 or more changed positions
    (4, 45, 7, 4, 7),
    (5, 40, 12, 5, 14),
    (6, 40, 13, 5, 21),
    (8, 60, 12, 4, 22),
    (4, 30, 14, 6, 23),
    (3, 25, 10, 6, 24),    # 2d > l with a deep tree
]


_DEEP_WANT = {}


@pytest.mark.parametrize("m", [4103, 4200])
def test_long_sequences_match_oracle(ctx, oracle_, m):
    # W = m - l + 1 = 4096 is the most windows the fused packing + masks kernel stages in
    # shared memory; at W = 4193 the plan takes the separate packing and masks kernels
    inst = pi.planted_instance(3, m, 8, 1, 40)
    want = oracle_.solve(inst.seqs, 8, 1, cap=1 << 24)
    got = ctx.solve(inst.seqs, 8, 1)
    assert len(want) > 30000
    assert np.array_equal(got, want)


def _window_keys(codes_row: np.ndarray, l: int) -> np.ndarray:
    # every l-mer of one sequence as its key (2 bits per base, position 0 most significant)
    k = np.zeros(len(codes_row) - l + 1, dtype=np.uint64)
    for p in range(l):
        k = (k << np.uint64(2)) | codes_row[p:p + len(k)].astype(np.uint64)
    return k


def test_maximum_sequence_length(ctx, oracle_):
    # m = 65536, the largest the boundary accepts. d = 0: the motifs are exactly the
    # l-mers common to both sequences (a set intersection). d = 1: sampled seeds
    # against the oracle, and the planted motif.
    l = 12
    inst = pi.planted_instance(2, 65536, l, 0, 41)
    codes = seq_codes(inst.seqs)
    want = np.intersect1d(_window_keys(codes[0], l), _window_keys(codes[1], l))
    assert np.array_equal(ctx.solve(inst.seqs, l, 0), want)
    inst = pi.planted_instance(2, 65536, l, 1, 42)
    got = ctx.solve(inst.seqs, l, 1)
    assert np.all(np.diff(got.astype(np.int64)) > 0)
    assert py_key(inst.motif.decode()) in set(int(k) for k in got)
    codes = seq_codes(inst.seqs[0])
    rng = np.random.default_rng(42)
    seeds = sorted(set(rng.choice(65536 - l + 1, size=5, replace=False).tolist()) | {int(inst.positions[0])})
    for j, w in oracle_per_seed(oracle_, inst.seqs, l, 1, seeds).items():
        assert np.array_equal(keys_within(got, codes[j:j + l], l, 1), w), j


@pytest.mark.parametrize("partial_rows", [-1, 1, 2, 5])
@pytest.mark.parametrize("case", DEEP, ids=lambda c: "n{}_m{}_l{}_d{}".format(*c[:4]))
def test_partial_level_matches_oracle(oracle_, case, partial_rows):
    # the partial-candidate level (letters fixed above the three lowest changed
    # positions, tested against the first rows before the leaves) off and on
    n, m, l, d, seed = case
    inst = pi.planted_instance(n, m, l, d, seed)
    seqs = pi.random_sequences(n, m, seed + 555)
    if case not in _DEEP_WANT:
        _DEEP_WANT[case] = (oracle_.solve(inst.seqs, l, d, cap=1 << 24), oracle_.solve(seqs, l, d, cap=1 << 24))
    want_planted, want_random = _DEEP_WANT[case]
    c = pms.Context(0)
    c.set_options(partial_rows=partial_rows)
    assert np.array_equal(c.solve(inst.seqs, l, d), want_planted)
    assert np.array_equal(c.solve(seqs, l, d), want_random)
    c.set_options(partial_rows=partial_rows, smem_rows=8)    # rows in global scratch
    assert np.array_equal(c.solve(inst.seqs, l, d), want_planted)
    c.close()


@pytest.mark.parametrize("l,d,partial_rows", [(13, 4, 3), (15, 4, 1), (17, 5, -1), (17, 5, 4)])
def test_partial_level_full_size_sampled_seeds(oracle_, l, d, partial_rows):
    c = pms.Context(0)
    c.set_options(partial_rows=partial_rows)
    _sampled_parity(c, oracle_, l, d, 2, 4)
    c.close()


@pytest.mark.parametrize("grab", [1, 32, 128])
@pytest.mark.parametrize("case", [c for c in SMALL if c[0] > 1] + DEEP, ids=lambda c: "n{}_m{}_l{}_d{}".format(*c[:4]))
def test_node_filter_modes_match_oracle(oracle_, case, grab):
    # grab = 1: lane-asynchronous node walk (the default); 32: guided node
    # batches; 128: fixed breadth-first batches of 128 nodes
    n, m, l, d, seed = case
    inst = pi.planted_instance(n, m, l, d, seed)
    want = oracle_.solve(inst.seqs, l, d, cap=1 << 24)
    c = pms.Context(0)
    c.set_options(grab=grab)
    assert np.array_equal(c.solve(inst.seqs, l, d), want)
    c.set_options(grab=grab, smem_rows=8)    # rows in global scratch
    assert np.array_equal(c.solve(inst.seqs, l, d), want)
    c.set_options(grab=grab, partial_rows=2)
    assert np.array_equal(c.solve(inst.seqs, l, d), want)
    c.close()


@pytest.mark.parametrize("l,d,grab", [(13, 4, 128), (15, 4, 1), (17, 5, 128), (15, 4, 32)])
def test_node_filter_modes_full_size_sampled_seeds(oracle_, l, d, grab):
    c = pms.Context(0)
    c.set_options(grab=grab)
    _sampled_parity(c, oracle_, l, d, 3, 4)
    c.close()


def test_plain_9_2_full_size_matches_oracle(ctx, oracle_):
    for seed in (1, 2, 3):
        inst = pi.plain_instance(9, 2, seed=seed)
        want = oracle_.solve(inst.seqs, 9, 2)
        got = ctx.solve(inst.seqs, 9, 2)
        assert np.array_equal(got, want)
        assert py_key(inst.motif.decode()) in set(int(k) for k in got)


def _sampled_parity(ctx, o, l, d, seed, nseeds):
    inst = pi.plain_instance(l, d, seed=seed)
    got = ctx.solve(inst.seqs, l, d)
    assert np.all(np.diff(got.astype(np.int64)) > 0) or len(got) <= 1   # sorted, unique
    assert py_key(inst.motif.decode()) in set(int(k) for k in got)
    for k in got:
        assert o.is_motif(o.decode(int(k), l), inst.seqs, d)
    W = inst.m - l + 1
    rng = np.random.default_rng(seed)
    seeds = set(rng.choice(W, size=nseeds, replace=False).tolist())
    seeds.add(int(inst.positions[0]))          # the seed at the planted copy in s_1
    want = oracle_per_seed(o, inst.seqs, l, d, sorted(seeds))
    codes = seq_codes(inst.seqs[0])
    for j, w in want.items():
        mine = keys_within(got, codes[j:j + l], l, d)
        assert np.array_equal(mine, w), (j, len(mine), len(w))
    return got


@pytest.mark.parametrize("l,d,seed,nseeds", [(11, 3, 1, 24), (13, 4, 1, 12), (15, 4, 1, 12), (15, 4, 2, 6),
                                               (17, 5, 1, 6)])
def test_plain_full_size_sampled_seeds(ctx, oracle_, l, d, seed, nseeds):
    _sampled_parity(ctx, oracle_, l, d, seed, nseeds)


def test_plain_19_6_full_size_sampled_seeds(ctx, oracle_):
    _sampled_parity(ctx, oracle_, 19, 6, 1, 1)


def test_device_entry_point_matches_host(ctx):
    import torch
    inst = pi.plain_instance(15, 4, seed=3)
    want = ctx.solve(inst.seqs, 15, 4)
    d_seqs = torch.from_numpy(inst.seqs.copy()).cuda()
    out = torch.zeros(1024, dtype=torch.int64, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    ctx.set_stream(torch.cuda.current_stream())
    ctx.solve_device(d_seqs, 20, 600, 15, 4, out, 1024, status)
    torch.cuda.synchronize()
    st = status.cpu().numpy().astype(np.uint32)
    assert st[2] == 0
    got = out[: int(st[1])].cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, want)
    ctx.set_stream(None)


def test_batch_matches_plain(ctx):
    insts = pi.batch_instances(count=24)
    res = ctx.solve_batch([(i.seqs, i.l, i.d) for i in insts])
    for i, r in zip(insts, res):
        assert not isinstance(r, Exception), r
        assert np.array_equal(r, ctx.solve(i.seqs, i.l, i.d))
        assert py_key(i.motif.decode()) in set(int(k) for k in r)


def test_batch_with_bad_instance(ctx):
    good = pi.plain_instance(9, 2, seed=5)
    bad = good.seqs.copy()
    bad[3, 7] = ord("N")
    res = ctx.solve_batch([(good.seqs, 9, 2), (bad, 9, 2), (good.seqs, 9, 9)])
    assert np.array_equal(res[0], ctx.solve(good.seqs, 9, 2))
    assert isinstance(res[1], pms.PMSError) and res[1].code == pms.PMS_EINVAL
    assert isinstance(res[2], pms.PMSError) and res[2].code == pms.PMS_EINVAL


def test_errors(ctx):
    inst = pi.plain_instance(9, 2, seed=1)
    bad = inst.seqs.copy()
    bad[0, 0] = ord("a")
    with pytest.raises(pms.PMSError) as e:
        ctx.solve(bad, 9, 2)
    assert e.value.code == pms.PMS_EINVAL
    for (l, d) in [(0, 0), (9, 9), (33, 2), (601, 1), (9, -1)]:
        with pytest.raises(pms.PMSError):
            ctx.solve(inst.seqs, l, d)
    # empty input (n = 0), sequences shorter than l, more sequences than the boundary takes
    for seqs, l in [(np.zeros((0, 40), np.uint8), 9), (inst.seqs[:, :8], 9), (np.full((65, 20), ord("A"), np.uint8), 5)]:
        with pytest.raises(pms.PMSError) as e:
            ctx.solve(seqs, l, 1)
        assert e.value.code == pms.PMS_EINVAL
    # device path reports an invalid byte in its status flags
    import torch
    d_seqs = torch.from_numpy(bad).cuda()
    out = torch.zeros(64, dtype=torch.int64, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    ctx.set_stream(torch.cuda.current_stream())
    ctx.solve_device(d_seqs, 20, 600, 9, 2, out, 64, status)
    torch.cuda.synchronize()
    ctx.set_stream(None)
    assert int(status[2].item()) & 1


@pytest.mark.parametrize("n,m,l,d,i,k", [(20, 600, 9, 2, 0, 0), (20, 600, 9, 2, 19, 599), (20, 600, 15, 4, 7, 300),
                                         (1, 40, 8, 2, 0, 39), (3, 17, 17, 3, 2, 16)])
def test_invalid_byte_found_anywhere(ctx, n, m, l, d, i, k):
    # the packing kernels find the byte; the host then names it
    seqs = pi.random_sequences(n, m, 11)
    bad = seqs.copy()
    bad[i, k] = ord("N")
    with pytest.raises(pms.PMSError) as e:
        ctx.solve(bad, l, d)
    assert e.value.code == pms.PMS_EINVAL
    assert f"byte {i * m + k} (0x4e)" in str(e.value)
    # the context stays usable
    assert np.array_equal(ctx.solve(seqs, l, d), ctx.solve(seqs.copy(), l, d))


def test_too_many_motifs_reported(ctx):
    c = pms.Context(0)
    c.set_options(max_motifs=16)
    seqs = pi.random_sequences(1, 30, 5)     # n = 1: B(x, 2) of 22 seeds, far more than 16
    with pytest.raises(pms.PMSError) as e:
        c.solve(seqs, 8, 2)
    assert e.value.code == pms.PMS_ETOOMANY
    c.close()


def test_work_counters(ctx):
    inst = pi.plain_instance(13, 4, seed=2)
    c = pms.Context(0)
    c.set_options(count_work=1)
    got = c.solve(inst.seqs, 13, 4)
    s = c.stats()
    assert np.array_equal(got, ctx.solve(inst.seqs, 13, 4))
    W = 600 - 13 + 1
    import math
    nsub = sum(math.comb(13, i) for i in range(5))
    assert s["candidates"] == W * sum(math.comb(13, i) * 3 ** i for i in range(5))
    assert s["subsets"] == (W - s["seeds_infeasible"]) * nsub
    assert s["cmp_rows"] >= W * 19 * (600 - 13 + 1)
    assert 0 < s["subsets_pruned"] < s["subsets"]
    c.close()


@pytest.mark.parametrize("triple_rows", [1, 3, 63])
@pytest.mark.parametrize("case", [c for c in SMALL if c[0] > 1] + DEEP, ids=lambda c: "n{}_m{}_l{}_d{}".format(*c[:4]))
def test_three_string_node_test_matches_oracle(oracle_, case, triple_rows):
    # the three-string test below a node (pivot occurrences kept only with a
    # feasible partner in each of the next triple_rows rows) on its own, with
    # the partial level, and with rows in global scratch
    n, m, l, d, seed = case
    inst = pi.planted_instance(n, m, l, d, seed)
    seqs = pi.random_sequences(n, m, seed + 991)
    want = oracle_.solve(inst.seqs, l, d, cap=1 << 24)
    c = pms.Context(0)
    c.set_options(triple_rows=triple_rows)
    assert np.array_equal(c.solve(inst.seqs, l, d), want)
    assert np.array_equal(c.solve(seqs, l, d), oracle_.solve(seqs, l, d, cap=1 << 24))
    c.set_options(triple_rows=triple_rows, partial_rows=2)
    assert np.array_equal(c.solve(inst.seqs, l, d), want)
    c.set_options(triple_rows=triple_rows, smem_rows=8)
    assert np.array_equal(c.solve(inst.seqs, l, d), want)
    c.close()
