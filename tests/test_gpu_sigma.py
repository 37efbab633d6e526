"""General alphabets (qPMS-Sigma) on the GPU through pms_solve_sigma, against the oracle.

Small instances: the motif set element by element against the oracle's full solve,
over alphabets of 2 to 32 letters, with quorums and the degenerate cases. Over
A, C, G, T: the DNA path. Full-size protein instances (n = 20, m = 600): sampled
seeds against the oracle, and properties that hold at any size (the planted
motif is found, every answer is a motif, the counters are exact).
"""
import numpy as np
import pytest

import planted_inputs as pi

pytestmark = pytest.mark.gpu

PROTEIN = pi.PROTEIN.decode()


def alphabet_of(sigma: int) -> str:
    return "".join(reversed("ACDEFGHIKLMNPQRSTVWYBJOUXZ0123456789"[:sigma]))


@pytest.fixture(scope="module")
def ctx():
    import paper_2403_00306_gb300 as pms
    c = pms.Context(0)
    yield c
    c.close()


SMALL = [
    # sigma, n, m, l, d, q, seed
    (2, 6, 40, 10, 2, 0, 1), (2, 4, 24, 12, 3, 3, 2), (3, 6, 50, 8, 2, 0, 3), (3, 5, 30, 7, 3, 4, 4),
    (4, 8, 60, 9, 2, 0, 5), (5, 6, 45, 7, 2, 0, 6), (7, 5, 40, 6, 2, 3, 7), (16, 6, 40, 6, 2, 0, 8),
    (17, 5, 30, 5, 2, 0, 9), (20, 8, 60, 7, 2, 0, 10), (20, 6, 50, 6, 3, 0, 11), (20, 5, 40, 6, 3, 3, 12),
    (20, 10, 100, 7, 3, 0, 13), (32, 4, 20, 4, 2, 0, 14), (32, 5, 30, 5, 2, 4, 15),
    (20, 1, 9, 5, 2, 0, 16),    # n = 1: the union of the spheres of the windows
    (20, 6, 30, 4, 0, 0, 17),   # d = 0: common l-mers
    (5, 4, 6, 6, 3, 0, 18),     # m = l: one window per sequence
    (20, 7, 33, 32, 1, 0, 19),  # l = 32: the whole plane word
    (2, 20, 800, 8, 4, 0, 20),  # every window is a row: more rows than shared memory holds
]


@pytest.mark.parametrize("sigma,n,m,l,d,q,seed", SMALL)
def test_small_instances_match_the_oracle(ctx, oracle_, sigma, n, m, l, d, q, seed):
    alpha = alphabet_of(sigma)
    inst = pi.planted_instance_sigma(n, m, l, d, seed, alpha.encode())
    want = oracle_.sigma_solve(inst.seqs, l, d, alpha, q=q, cap=1 << 22)
    got = ctx.solve_sigma(inst.seqs, l, d, alpha, q=q)
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.array_equal(got, want)
    assert inst.motif.decode() in {bytes(r).decode() for r in got}


def test_random_backgrounds_match_the_oracle(ctx, oracle_):
    rng = np.random.default_rng(77)
    for sigma, n, m, l, d in [(20, 6, 40, 6, 3), (3, 8, 60, 9, 3), (32, 3, 25, 5, 2), (2, 10, 50, 12, 3)]:
        alpha = alphabet_of(sigma)
        letters = np.frombuffer(alpha.encode(), np.uint8)
        seqs = letters[rng.integers(0, sigma, size=(n, m))].astype(np.uint8)
        for q in (0, n - 1):
            want = oracle_.sigma_solve(seqs, l, d, alpha, q=q, cap=1 << 22)
            assert np.array_equal(ctx.solve_sigma(seqs, l, d, alpha, q=q), want), (sigma, n, m, l, d, q)


@pytest.mark.parametrize("l,d", [(9, 2), (13, 4), (15, 4)])
def test_acgt_equals_the_dna_path(ctx, oracle_, l, d):
    # over A, C, G, T the general search must return the DNA search's motifs
    inst = pi.planted_instance(20, 600, l, d, 3)
    codes = ctx.solve(inst.seqs, l, d)
    want = [oracle_.decode(int(k), l) for k in codes]
    got = [bytes(r).decode() for r in ctx.solve_sigma(inst.seqs, l, d, "ACGT")]
    assert got == want
    if (l, d) == (9, 2):
        assert want == [oracle_.decode(int(k), l) for k in oracle_.solve(inst.seqs, l, d)]


def test_acgt_quorum_equals_the_dna_quorum(ctx, oracle_):
    inst = pi.planted_instance(12, 200, 11, 3, 5)
    want = [oracle_.decode(int(k), 11) for k in oracle_.solve_quorum(inst.seqs, 11, 3, 9)]
    got = [bytes(r).decode() for r in ctx.solve_sigma(inst.seqs, 11, 3, "ACGT", q=9)]
    assert got == want


@pytest.mark.parametrize("l,d", [(9, 3), (11, 4), (9, 4)])
def test_full_size_protein(ctx, oracle_, l, d):
    n, m = 20, 600
    inst = pi.planted_instance_sigma(n, m, l, d, 1)
    got = ctx.solve_sigma(inst.seqs, l, d, PROTEIN)
    found = [bytes(r).decode() for r in got]
    assert inst.motif.decode() in found
    for s in found:
        assert oracle_.is_motif(s, inst.seqs, d)
    st = ctx.stats()
    W = m - l + 1
    # every seed compares itself with every window of the other sequences once
    assert st["cmp_rows"] == W * (n - 1) * W
    nodes = sum(__import__("math").comb(l, k) for k in range(d + 1))
    assert st["subsets"] == (W - st["seeds_infeasible"]) * nodes
    assert 0 <= st["subsets_pruned"] <= st["subsets"]
    # the same answer from one CTA per SM (another interleaving of the seed queue)
    ctx.set_options(ctas_per_sm=1)
    try:
        assert np.array_equal(ctx.solve_sigma(inst.seqs, l, d, PROTEIN), got)
    finally:
        ctx.set_options(ctas_per_sm=0)
    if (l, d) == (9, 3):
        # sampled seeds against the oracle: the planted copy in s_1 and a few more
        p0 = int(inst.positions[0])
        for lo, hi in [(p0, p0 + 1), (0, 4), (W - 4, W)]:
            want = {bytes(r).decode() for r in oracle_.sigma_solve_seeds(inst.seqs, l, d, PROTEIN, lo, hi)}
            near = {s for s in found
                    if any(sum(a != b for a, b in zip(s, bytes(inst.seqs[0, j:j + l]).decode())) <= d
                           for j in range(lo, hi))}
            assert near == want, (lo, hi)


def test_overflow_grows_once_then_reports(ctx, oracle_):
    import paper_2403_00306_gb300 as pms
    # n = 1 over 32 letters: every string within 3 of one of the three windows
    seqs = np.frombuffer(b"ABCDEFGH", np.uint8).reshape(1, 8)
    alpha = "ABCDEFGHIJKLMNOPQRSTUVWXYZ012345"
    want = oracle_.sigma_solve(seqs, 6, 3, alpha, cap=1 << 22)
    got = ctx.solve_sigma(seqs, 6, 3, alpha)          # 1.8 million raw keys: the buffer grows once
    assert np.array_equal(got, want)
    ctx.set_options(max_motifs=1024)
    try:
        with pytest.raises(pms.PMSError) as e:
            ctx.solve_sigma(seqs, 6, 3, alpha)
        assert e.value.code == pms.PMS_ETOOMANY
    finally:
        ctx.set_options(max_motifs=0)


def test_large_output_with_keys_over_two_words(ctx, oracle_):
    # n = 1 over the twenty amino acids, l = 16: keys of 80 bits (two of the three words),
    # about 130,000 raw keys, so the sort takes its radix form
    rng = np.random.default_rng(11)
    seqs = np.frombuffer(bytes(rng.choice(np.frombuffer(PROTEIN.encode(), np.uint8), 18)), np.uint8).reshape(1, 18)
    want = oracle_.sigma_solve(seqs, 16, 2, PROTEIN, cap=1 << 22)
    got = ctx.solve_sigma(seqs, 16, 2, PROTEIN)
    assert len(want) > 100000
    assert np.array_equal(got, want)


@pytest.mark.parametrize("alpha,seq,l,d", [
    ("ACGT", "A" * 20, 8, 3),          # 13 equal windows: 23,257 raw keys, each value 13 times, across CTA tiles
    ("ACDEF", None, 7, 2),             # 13 windows: 4,745 raw keys, just above the one-CTA network's 4,096
    ("ACDEFGHIKLMNPQRSTVWY", "ACACACACACACACACAC", 9, 2),   # two window kinds, five times each
])
def test_sort_across_the_grid(ctx, oracle_, alpha, seq, l, d):
    # n = 1: the motif set is the union of the windows' spheres; the raw keys exceed what
    # one CTA's network sorts, so every CTA of the sort takes a tile
    if seq is None:
        rng = np.random.default_rng(5)
        seq = bytes(rng.choice(np.frombuffer(alpha.encode(), np.uint8), 19)).decode()
    seqs = np.frombuffer(seq.encode(), np.uint8).reshape(1, -1)
    want = oracle_.sigma_solve(seqs, l, d, alpha, cap=1 << 22)
    got = ctx.solve_sigma(seqs, l, d, alpha)
    assert np.array_equal(got, want)


def test_invalid_inputs(ctx):
    import paper_2403_00306_gb300 as pms
    inst = pi.planted_instance_sigma(4, 30, 6, 2, 3)
    bad = inst.seqs.copy()
    bad[2, 7] = ord("B")   # not an amino-acid letter
    cases = [
        dict(seqs=bad, l=6, d=2, alphabet=PROTEIN),
        dict(seqs=inst.seqs, l=6, d=2, alphabet="AACDE"),        # repeated letter
        dict(seqs=inst.seqs, l=6, d=2, alphabet="A"),            # one letter
        dict(seqs=inst.seqs, l=6, d=2, alphabet=PROTEIN + "BJOUXZ0123456789"),   # 36 letters
        dict(seqs=inst.seqs, l=6, d=6, alphabet=PROTEIN),        # d >= l
        dict(seqs=inst.seqs, l=40, d=2, alphabet=PROTEIN),       # l > 32
        dict(seqs=inst.seqs, l=6, d=2, alphabet=PROTEIN, q=5),   # q > n
    ]
    for kw in cases:
        with pytest.raises(pms.PMSError) as e:
            ctx.solve_sigma(**kw)
        assert e.value.code == pms.PMS_EINVAL, kw
    # the context stays usable
    assert inst.motif.decode() in {bytes(r).decode() for r in ctx.solve_sigma(inst.seqs, 6, 2, PROTEIN)}


def test_capped_grid_matches_the_oracle(oracle_, monkeypatch):
    # rows beyond shared memory go to a per-CTA global scratch whose total is capped
    # (2 GiB; lowered here through PMS_SIGMA_SCRATCH_CAP so that only a few CTAs run)
    import paper_2403_00306_gb300 as pms
    sigma, n, m, l, d = 2, 20, 800, 8, 4
    alpha = alphabet_of(sigma)
    inst = pi.planted_instance_sigma(n, m, l, d, 20, alpha.encode())
    want = oracle_.sigma_solve(inst.seqs, l, d, alpha, cap=1 << 22)
    per_cta = 4 * 2 * (n - 1) * (m - l + 1)          # D words and one plane per row
    monkeypatch.setenv("PMS_SIGMA_SCRATCH_CAP", str(3 * per_cta))   # three CTAs
    c = pms.Context(0)
    assert np.array_equal(c.solve_sigma(inst.seqs, l, d, alpha), want)
    monkeypatch.delenv("PMS_SIGMA_SCRATCH_CAP")
    assert np.array_equal(c.solve_sigma(inst.seqs, l, d, alpha), want)
    c.close()
