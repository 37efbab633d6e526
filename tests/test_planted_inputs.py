"""The seeded input generators: the counter-based SplitMix64 stream, the bounded and
unit maps, and the FM planting rule of the paper's experiments (one copy of the motif
per string, exactly d substitutions at distinct positions, each to another base)."""
import numpy as np
import pytest

from planted_inputs import (ALPHABET, batch_instances, bounded, planted_instance,
                            random_sequences, serve_requests, splitmix64, unit_float)

M64 = (1 << 64) - 1


def splitmix64_int(state):
    # the generator's published definition, in Python integers: add the golden
    # gamma, then the two xor-shift-multiply rounds and a final xor-shift
    state = (state + 0x9E3779B97F4A7C15) & M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return state, z ^ (z >> 31)


def test_stream_zero_is_the_sequential_generator_seeded_with_zero():
    # the first outputs of SplitMix64 seeded with 0, as its reference implementation prints them
    known = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
             0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [int(x) for x in splitmix64(0, range(5))] == known


def test_counter_form_equals_the_sequential_form():
    for stream in (1, 12345, M64 - 7):
        state, seq = stream, []
        for _ in range(64):
            state, z = splitmix64_int(state)
            seq.append(z)
        assert [int(x) for x in splitmix64(stream, range(64))] == seq
        # any counter subset draws the same values as the full sequence
        assert [int(x) for x in splitmix64(stream, [63, 0, 17])] == [seq[63], seq[0], seq[17]]


def test_bounded_and_unit_maps():
    u = splitmix64(99, range(20000))
    for r in (1, 3, 7, 600):
        v = bounded(u, r)
        assert v.min() >= 0 and v.max() < r
        ref = [((int(x) >> 32) * r) >> 32 for x in u[:50]]
        assert [int(x) for x in v[:50]] == ref
    assert set(int(x) for x in bounded(u, 3)) == {0, 1, 2}
    f = unit_float(u)
    assert f.min() >= 0.0 and f.max() < 1.0
    assert abs(f.mean() - 0.5) < 0.01
    assert unit_float(np.array([M64], dtype=np.uint64))[0] < 1.0


def hamming(a, b):
    return int(np.count_nonzero(np.frombuffer(a, np.uint8) != np.frombuffer(b, np.uint8)))


@pytest.mark.parametrize("n,m,l,d,seed", [(20, 600, 15, 4, 1), (5, 40, 9, 2, 3), (3, 12, 12, 5, 8),
                                          (4, 30, 7, 0, 2), (2, 20, 6, 6, 5)])
def test_planting_rule(n, m, l, d, seed):
    inst = planted_instance(n, m, l, d, seed)
    assert inst.seqs.shape == (n, m) and inst.seqs.dtype == np.uint8
    assert set(inst.seqs.tobytes()) <= set(ALPHABET)
    assert len(inst.motif) == l and set(inst.motif) <= set(ALPHABET)
    assert (inst.n, inst.m, inst.l, inst.d) == (n, m, l, d)
    for i in range(n):
        p = int(inst.positions[i])
        assert 0 <= p <= m - l
        # exactly d distinct positions changed, each to a different base
        assert hamming(inst.seqs[i, p:p + l].tobytes(), inst.motif) == d


def test_generators_are_deterministic_and_seed_dependent():
    a = planted_instance(10, 200, 13, 4, 7)
    b = planted_instance(10, 200, 13, 4, 7)
    c = planted_instance(10, 200, 13, 4, 8)
    assert np.array_equal(a.seqs, b.seqs) and a.motif == b.motif
    assert np.array_equal(a.positions, b.positions)
    assert not np.array_equal(a.seqs, c.seqs)
    assert np.array_equal(random_sequences(4, 50, 3), random_sequences(4, 50, 3))


def test_background_bases_are_uniform():
    s = random_sequences(50, 2000, 11)
    counts = np.array([np.count_nonzero(s == ch) for ch in ALPHABET])
    assert counts.sum() == s.size
    # four equally likely bases: each share within 1% of a quarter
    assert np.all(np.abs(counts / s.size - 0.25) < 0.01)


def test_substituted_bases_are_the_three_others_uniformly():
    # over many planted copies, each changed position carries each of the three
    # other bases about equally often
    counts = np.zeros((4, 4), dtype=np.int64)
    for seed in range(40):
        inst = planted_instance(30, 40, 12, 4, seed)
        motif = np.frombuffer(inst.motif, np.uint8)
        for i in range(inst.n):
            p = int(inst.positions[i])
            copy = inst.seqs[i, p:p + inst.l]
            for k in np.nonzero(copy != motif)[0]:
                counts[ALPHABET.index(motif[k]), ALPHABET.index(copy[k])] += 1
    assert np.all(np.diag(counts) == 0)
    for a in range(4):
        row = counts[a][[b for b in range(4) if b != a]]
        assert row.sum() > 0
        assert np.all(np.abs(row / row.sum() - 1 / 3) < 0.06)


def test_parameter_errors():
    for args in ((0, 10, 3, 1), (2, 10, 11, 1), (2, 10, 3, 4), (2, 10, 3, -1), (2, 10, 0, 0)):
        with pytest.raises(ValueError):
            planted_instance(*args, seed=1)


def test_batch_and_served_workloads_follow_their_ranges():
    insts = batch_instances(40, master_seed=5)
    assert len(insts) == 40
    for inst in insts:
        assert (inst.l, inst.d) in ((11, 3), (13, 4), (15, 4))
        assert 10 <= inst.n <= 30 and 300 <= inst.m <= 1000
    assert [i.seed for i in insts] == [i.seed for i in batch_instances(40, master_seed=5)]
    reqs = list(serve_requests(300, rate_per_s=100.0, master_seed=3))
    times = np.array([t for t, _ in reqs])
    assert np.all(np.diff(times) > 0)
    # Poisson arrivals at 100/s: mean gap 10 ms
    assert abs(np.mean(np.diff(times)) - 0.01) < 0.002
    for _, inst in reqs[:20]:
        assert inst.n == 20 and 200 <= inst.m <= 1200 and (inst.l, inst.d) in ((13, 4), (15, 4), (17, 5))


@pytest.mark.parametrize("alphabet,l,d,seed", [(b"ACDEFGHIKLMNPQRSTVWY", 11, 4, 1), (b"01", 8, 3, 2),
                                                (b"ACG", 6, 6, 3), (b"ACDEFGHIKLMNPQRSTVWY", 9, 0, 4)])
def test_planting_rule_over_a_general_alphabet(alphabet, l, d, seed):
    from planted_inputs import planted_instance_sigma
    inst = planted_instance_sigma(12, 80, l, d, seed, alphabet)
    assert set(inst.seqs.tobytes()) <= set(alphabet) and set(inst.motif) <= set(alphabet)
    for i in range(inst.n):
        p = int(inst.positions[i])
        assert hamming(inst.seqs[i, p:p + l].tobytes(), inst.motif) == d
    again = planted_instance_sigma(12, 80, l, d, seed, alphabet)
    assert np.array_equal(inst.seqs, again.seqs) and inst.motif == again.motif


def test_protein_background_uses_every_letter_uniformly():
    from planted_inputs import PROTEIN, planted_instance_sigma
    s = planted_instance_sigma(40, 1000, 5, 0, 9).seqs
    counts = np.array([np.count_nonzero(s == ch) for ch in PROTEIN])
    assert np.all(np.abs(counts / s.size - 1 / 20) < 0.005)
    with pytest.raises(ValueError):
        planted_instance_sigma(2, 10, 3, 1, 1, b"AA")
