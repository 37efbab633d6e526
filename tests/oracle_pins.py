"""Checks that pin the CPU oracle to facts fixed outside it.

Each check takes an ``oracle.Oracle`` and raises AssertionError on failure, so
the same checks run against the real oracle (test_oracle.py) and against
copies of it with a planted mistake (test_oracle_mutants.py). None of them
re-types the oracle's own arithmetic: they use the paper's printed worked
example, closed-form counts, exhaustive enumeration written independently in
Python, and invariants of the problem definition.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np

import planted_inputs as pi

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ACGT = "ACGT"


def n_ball(l: int, d: int) -> int:
    """|B(x, d)| for an l-mer over a 4-letter alphabet: choose i positions, 3 other letters each."""
    return sum(math.comb(l, i) * 3 ** i for i in range(d + 1))


def pair_ball_size(l: int, d: int, D: int) -> int:
    """|B(x,d) & B(r,d)| when d_H(x,r) = D, counted by classes.

    Of the l - D positions where x and r agree, a are changed (3 letters
    each); of the D positions where they differ, t take a third letter
    (2 each), e_x keep x's letter and the rest take r's letter. The distance
    to x is a + t + (D - t - e_x), to r it is a + t + e_x.
    """
    total = 0
    for a in range(l - D + 1):
        for t in range(D + 1):
            for ex in range(D - t + 1):
                er = D - t - ex
                if a + t + er <= d and a + t + ex <= d:
                    total += math.comb(l - D, a) * 3 ** a * math.comb(D, t) * 2 ** t * math.comb(D - t, ex)
    return total


def py_hamming(a: str, b: str) -> int:
    return sum(x != y for x, y in zip(a, b))


def py_key(s: str) -> int:
    k = 0
    for ch in s:
        k = 4 * k + ACGT.index(ch)
    return k


def lmers(seq: bytes, l: int) -> set[str]:
    s = seq.decode() if isinstance(seq, (bytes, bytearray)) else bytes(seq).decode()
    return {s[j:j + l] for j in range(len(s) - l + 1)}


def read_compression_golden():
    lm, pairs, misprint = {}, [], {}
    with open(os.path.join(GOLDEN, "compression_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "lmer":
                lm[tok[1]] = dict(codes=tok[2], group1=tok[3], group0=tok[4])
            elif tok[0] == "pair":
                pairs.append(dict(a=tok[1], b=tok[2], xor1=tok[3], xor0=tok[4], orr=tok[5], setbits=int(tok[6])))
            elif tok[0] == "misprint":
                misprint[(tok[1], tok[2])] = tok[3]
    return lm, pairs, misprint


def plane_string(word: int, l: int) -> str:
    """Bits 0..l-1 of a plane word printed position 1 first, as the paper prints them."""
    return "".join("1" if (word >> k) & 1 else "0" for k in range(l))


# --------------------------------------------------------------------------- pins

def check_compression_example(o) -> None:
    lm, pairs, misprint = read_compression_golden()
    for s, row in lm.items():
        planes = o.compress(s)
        l = len(s)
        g0, g1 = plane_string(int(planes[0, 0]), l), plane_string(int(planes[1, 0]), l)
        want1 = misprint.get((s, "group1"), row["group1"])
        assert g1 == want1, (s, g1, want1)
        assert g0 == row["group0"], (s, g0, row["group0"])
        # the printed codes column, group1*2 + group0 per position
        codes = "".join(str(2 * int(a) + int(b)) for a, b in zip(g1, g0))
        assert codes == row["codes"], (s, codes)
    for p in pairs:
        a, b = o.compress(p["a"]), o.compress(p["b"])
        l = len(p["a"])
        assert o.compressed_distance(a, b, l) == p["setbits"]
        assert o.hamming(p["a"], p["b"]) == p["setbits"]
        x1 = plane_string(int(a[1, 0] ^ b[1, 0]), l)
        x0 = plane_string(int(a[0, 0] ^ b[0, 0]), l)
        assert x0 == p["xor0"]
        assert plane_string(int((a[1, 0] ^ b[1, 0]) | (a[0, 0] ^ b[0, 0])), l) == p["orr"]
        # the printed xor1 is the xor with the misprinted group1 of b
        printed_g1_b = int(lm[p["b"]]["group1"][::-1], 2)
        assert plane_string(int(a[1, 0]) ^ printed_g1_b, l) == p["xor1"]
        assert x1 != p["xor1"]


def check_distance_definitions(o) -> None:
    rng = np.random.default_rng(5)
    for _ in range(200):
        l = int(rng.integers(1, 12))
        a = "".join(rng.choice(list(ACGT), l))
        b = "".join(rng.choice(list(ACGT), l))
        assert o.hamming(a, b) == py_hamming(a, b)
        pa, pb = o.compress(a), o.compress(b)
        assert o.compressed_distance(pa, pb, l) == py_hamming(a, b)
        m = l + int(rng.integers(0, 8))
        s = "".join(rng.choice(list(ACGT), m))
        want = min(py_hamming(a, s[j:j + l]) for j in range(m - l + 1))
        assert o.distance_to_string(a, s) == want
    # multi-word planes (l > 32): the compressed distance still equals Definition 3
    for l in (33, 40, 64):
        a = "".join(rng.choice(list(ACGT), l))
        b = "".join(rng.choice(list(ACGT), l))
        assert o.compressed_distance(o.compress(a), o.compress(b), l) == py_hamming(a, b)


def check_neighbourhood_counts(o) -> None:
    rng = np.random.default_rng(11)
    for (l, d) in [(1, 0), (1, 1), (5, 0), (6, 2), (9, 2), (11, 3), (13, 4), (15, 4)]:
        x = "".join(rng.choice(list(ACGT), l))
        nb = o.neighbourhood(x, d)
        assert len(nb) == n_ball(l, d), (l, d, len(nb))
        assert o.neighbourhood_visits(x, d) == n_ball(l, d)
    for (l, d) in [(17, 5), (19, 6)]:
        x = "".join(rng.choice(list(ACGT), l))
        assert o.neighbourhood_visits(x, d) == n_ball(l, d)


def check_neighbourhood_members(o) -> None:
    rng = np.random.default_rng(12)
    for (l, d) in [(4, 1), (5, 2), (6, 3), (6, 6)]:
        x = "".join(rng.choice(list(ACGT), l))
        want = sorted(py_key("".join(t)) for t in itertools.product(ACGT, repeat=l)
                      if py_hamming(x, "".join(t)) <= d)
        got = [int(k) for k in o.neighbourhood(x, d)]
        assert got == want, (l, d)


def check_pair_intersections(o) -> None:
    rng = np.random.default_rng(13)
    for (l, d) in [(8, 2), (10, 3), (11, 3)]:
        for D in range(0, 2 * d + 2):
            x = list(rng.choice(list(ACGT), l))
            r = list(x)
            for p in rng.choice(l, size=min(D, l), replace=False):
                r[p] = ACGT[(ACGT.index(r[p]) + 1 + int(rng.integers(0, 3))) % 4]
            xs, rs = "".join(x), "".join(r)
            assert py_hamming(xs, rs) == min(D, l)
            got = o.pair_intersection_size(xs, rs, d)
            want = pair_ball_size(l, d, min(D, l)) if D <= 2 * d else 0
            assert got == want, (l, d, D, got, want)


def check_bruteforce_agreement(o) -> None:
    cases = [(3, 20, 5, 1, 101), (4, 24, 6, 1, 102), (5, 30, 6, 2, 103), (6, 40, 7, 2, 104),
             (4, 16, 4, 2, 105), (2, 12, 5, 3, 106), (6, 25, 8, 2, 107), (1, 9, 5, 2, 108)]
    for (n, m, l, d, seed) in cases:
        inst = pi.planted_instance(n, m, l, d, seed)
        bf = o.bruteforce(inst.seqs, l, d)
        a = o.solve(inst.seqs, l, d, threads=2)
        assert np.array_equal(a, bf), (n, m, l, d, seed)
        b = o.solve_pairs(inst.seqs, l, d, threads=2)
        assert np.array_equal(b, bf), (n, m, l, d, seed)
        seqs = pi.random_sequences(n, m, seed + 1000)
        assert np.array_equal(o.solve(seqs, l, d, threads=2), o.bruteforce(seqs, l, d))


def check_planted_motif_found(o) -> None:
    for (l, d, seed) in [(9, 2, 1), (9, 2, 2), (9, 2, 3), (8, 1, 4), (10, 3, 5)]:
        inst = pi.planted_instance(20, 120, l, d, seed)
        got = o.solve(inst.seqs, l, d)
        assert py_key(inst.motif.decode()) in set(int(k) for k in got), (l, d, seed)
        for k in got[:50]:
            assert o.is_motif(o.decode(int(k), l), inst.seqs, d)


def check_special_cases(o) -> None:
    # d = 0: the motifs are the l-mers present in every sequence
    for seed in range(3):
        inst = pi.planted_instance(4, 30, 5, 0, 200 + seed)
        sets = [lmers(bytes(row), 5) for row in inst.seqs]
        want = sorted(py_key(s) for s in set.intersection(*sets))
        assert [int(k) for k in o.solve(inst.seqs, 5, 0, threads=1)] == want
    # n = 1: every string within d of some l-mer of the single sequence
    seqs = pi.random_sequences(1, 12, 300)
    l, d = 5, 1
    want = set()
    for x in lmers(bytes(seqs[0]), l):
        for t in itertools.product(ACGT, repeat=l):
            s = "".join(t)
            if py_hamming(x, s) <= d:
                want.add(py_key(s))
    assert [int(k) for k in o.solve(seqs, l, d, threads=1)] == sorted(want)


def check_invariants(o) -> None:
    inst = pi.planted_instance(8, 60, 7, 2, 400)
    base = set(int(k) for k in o.solve(inst.seqs, 7, 2, threads=2))
    # monotone in d
    for d in range(0, 3):
        lo = set(int(k) for k in o.solve(inst.seqs, 7, d, threads=2))
        hi = set(int(k) for k in o.solve(inst.seqs, 7, d + 1, threads=2))
        assert lo <= hi
    # permuting the sequences changes nothing
    perm = inst.seqs[np.random.default_rng(3).permutation(8)]
    assert set(int(k) for k in o.solve(perm, 7, 2, threads=2)) == base
    # one sequence more can only remove motifs
    extra = np.vstack([inst.seqs, pi.random_sequences(1, 60, 401)])
    assert set(int(k) for k in o.solve(extra, 7, 2, threads=2)) <= base
    # seed slices partition the work
    parts = set()
    for lo in range(0, 54, 9):
        parts |= set(int(k) for k in o.solve_seeds(inst.seqs, 7, 2, lo, lo + 9, threads=1))
    assert parts == base


def check_quorum(o) -> None:
    # brute force with a quorum on tiny inputs, every q
    for (n, m, l, d, seed) in [(5, 30, 6, 1, 501), (4, 25, 5, 2, 502), (6, 20, 6, 2, 503)]:
        inst = pi.planted_instance(n, m, l, d, seed)
        prev = None
        for q in range(1, n + 1):
            got = o.solve_quorum(inst.seqs, l, d, q, threads=2)
            assert np.array_equal(got, o.bruteforce_quorum(inst.seqs, l, d, q)), (n, m, l, d, q)
            assert py_key(inst.motif.decode()) in set(int(k) for k in got)
            if prev is not None:
                assert set(int(k) for k in got) <= prev          # fewer motifs as the quorum rises
            prev = set(int(k) for k in got)
        # q = n is the PMS problem
        assert np.array_equal(o.solve_quorum(inst.seqs, l, d, n, threads=2), o.solve(inst.seqs, l, d, threads=2))
    # q = 1: every string within d of some l-mer of some sequence (written out in Python)
    seqs = pi.random_sequences(3, 9, 510)
    l, d = 5, 1
    want = set()
    for row in seqs:
        for x in lmers(bytes(row), l):
            for t in itertools.product(ACGT, repeat=l):
                s = "".join(t)
                if py_hamming(x, s) <= d:
                    want.add(py_key(s))
    assert [int(k) for k in o.solve_quorum(seqs, l, d, 1, threads=1)] == sorted(want)


def check_packed_solver(o) -> None:
    """The solver on compressed l-mers: brute force over 4^l, the definition written out in
    Python (d = 0, n = 1), the char-level solver on edge shapes, and seed slices partitioning."""
    cases = [(3, 20, 5, 1, 601), (5, 30, 6, 2, 602), (4, 16, 4, 2, 603), (1, 9, 5, 2, 604), (6, 25, 8, 2, 605)]
    for (n, m, l, d, seed) in cases:
        inst = pi.planted_instance(n, m, l, d, seed)
        assert np.array_equal(o.solve_packed(inst.seqs, l, d, threads=2), o.bruteforce(inst.seqs, l, d)), \
            (n, m, l, d)
        seqs = pi.random_sequences(n, m, seed + 1000)
        assert np.array_equal(o.solve_packed(seqs, l, d, threads=2), o.bruteforce(seqs, l, d))
    # d = 0: the l-mers present in every sequence
    inst = pi.planted_instance(4, 30, 5, 0, 610)
    want = sorted(py_key(s) for s in set.intersection(*[lmers(bytes(row), 5) for row in inst.seqs]))
    assert [int(k) for k in o.solve_packed(inst.seqs, 5, 0, threads=1)] == want
    # n = 1: every string within d of some l-mer of the single sequence
    seqs = pi.random_sequences(1, 11, 611)
    want = set()
    for x in lmers(bytes(seqs[0]), 5):
        for t in itertools.product(ACGT, repeat=5):
            if py_hamming(x, "".join(t)) <= 1:
                want.add(py_key("".join(t)))
    assert [int(k) for k in o.solve_packed(seqs, 5, 1, threads=1)] == sorted(want)
    # the char-level solver at l = 32, m = l, and on instances with many motifs
    for (n, m, l, d, seed) in [(3, 40, 32, 2, 612), (4, 9, 9, 3, 613), (20, 120, 9, 2, 614), (6, 60, 7, 2, 615),
                               (10, 80, 10, 3, 616)]:
        inst = pi.planted_instance(n, m, l, d, seed)
        want = o.solve(inst.seqs, l, d, threads=2)
        got = o.solve_packed(inst.seqs, l, d, threads=2)
        assert np.array_equal(got, want), (n, m, l, d, len(got), len(want))
        assert py_key(inst.motif.decode()) in set(int(k) for k in got)
    # seed slices partition the work
    inst = pi.planted_instance(8, 60, 7, 2, 617)
    parts = set()
    for lo in range(0, 54, 9):
        parts |= set(int(k) for k in o.solve_packed(inst.seqs, 7, 2, lo, lo + 9, threads=1))
    assert parts == set(int(k) for k in o.solve(inst.seqs, 7, 2, threads=2))
    parts = set()
    for lo in range(0, 54, 18):
        parts |= set(int(k) for k in o.solve_pairs_seeds(inst.seqs, 7, 2, lo, lo + 18, threads=1))
    assert parts == set(int(k) for k in o.solve(inst.seqs, 7, 2, threads=2))


# ------------------------------------------------------------- general alphabets (qPMS-Sigma)

PROTEIN = pi.PROTEIN.decode()


def n_ball_sigma(l: int, d: int, sigma: int) -> int:
    """|B(x, d)| over sigma letters: choose i positions, sigma - 1 other letters each."""
    return sum(math.comb(l, i) * (sigma - 1) ** i for i in range(d + 1))


def alphabet_of(sigma: int) -> str:
    # sigma distinct printable letters, deliberately not in ASCII order
    return "".join(reversed("ACDEFGHIKLMNPQRSTVWYBJOUXZ0123456789"[:sigma]))


def random_over(rng, alphabet: str, shape) -> np.ndarray:
    letters = np.frombuffer(alphabet.encode(), dtype=np.uint8)
    return letters[rng.integers(0, len(alphabet), size=shape)].astype(np.uint8)


def py_sigma_motifs(seqs: np.ndarray, l: int, d: int, alphabet: str, q: int = 0) -> list[str]:
    """Definition 5 over every string of alphabet^l, written out in Python (tiny cases only)."""
    rows = [bytes(r).decode() for r in seqs]
    need = q or len(rows)
    out = []
    for t in itertools.product(alphabet, repeat=l):
        s = "".join(t)
        hits = sum(1 for r in rows if any(py_hamming(s, r[j:j + l]) <= d for j in range(len(r) - l + 1)))
        if hits >= need:
            out.append(s)
    return out          # itertools.product yields the alphabet's index order


def as_strings(arr: np.ndarray) -> list[str]:
    return [bytes(r).decode() for r in arr]


def check_sigma_compression(o) -> None:
    # ceil(log2 sigma) groups
    assert [o.sigma_groups(s) for s in (2, 3, 4, 5, 8, 9, 16, 17, 20, 32)] == [1, 2, 2, 3, 3, 4, 4, 5, 5, 5]
    rng = np.random.default_rng(21)
    for sigma in (2, 3, 5, 17, 20, 32):
        alpha = alphabet_of(sigma)
        for _ in range(60):
            l = int(rng.integers(1, 33))
            a = bytes(random_over(rng, alpha, l)).decode()
            b = bytes(random_over(rng, alpha, l)).decode()
            pa, pb = o.sigma_compress(alpha, a), o.sigma_compress(alpha, b)
            assert pa.shape == (o.sigma_groups(sigma), 1)
            assert o.sigma_compressed_distance(pa, pb, l) == py_hamming(a, b), (sigma, a, b)
            # group g, bit k holds bit g of the index of letter k
            for k in (0, l - 1):
                idx = alpha.index(a[k])
                assert [(int(pa[g, 0]) >> k) & 1 for g in range(pa.shape[0])] == \
                    [(idx >> g) & 1 for g in range(pa.shape[0])]
    # over A, C, G, T the groups are the DNA planes of the paper's example
    for s in ("AGGCTA", "GAGCAT", "ACGTTGCA"):
        assert np.array_equal(o.sigma_compress(ACGT, s), o.compress(s))


def check_sigma_neighbourhood_counts(o) -> None:
    rng = np.random.default_rng(22)
    for sigma, l, d in [(2, 10, 3), (3, 8, 8), (5, 6, 3), (20, 7, 2), (20, 5, 4), (32, 4, 2), (4, 13, 4)]:
        alpha = alphabet_of(sigma)
        x = bytes(random_over(rng, alpha, l)).decode()
        assert o.sigma_neighbourhood_visits(alpha, x, d) == n_ball_sigma(l, d, sigma), (sigma, l, d)


def check_sigma_bruteforce(o) -> None:
    rng = np.random.default_rng(23)
    # the oracle's brute force against the definition written out in Python
    for sigma, n, m, l, d, q in [(3, 3, 8, 4, 1, 0), (5, 2, 7, 3, 1, 0), (2, 4, 9, 5, 1, 3), (20, 2, 5, 2, 1, 0)]:
        alpha = alphabet_of(sigma)
        seqs = random_over(rng, alpha, (n, m))
        want = py_sigma_motifs(seqs, l, d, alpha, q)
        assert as_strings(o.sigma_bruteforce(seqs, l, d, alpha, q=q)) == want, (sigma, n, m, l, d, q)
        assert as_strings(o.sigma_solve(seqs, l, d, alpha, q=q, threads=1)) == want, (sigma, n, m, l, d, q)
    # the tree search against the brute force on planted and random inputs, every quorum
    for sigma, n, m, l, d, seed in [(2, 4, 20, 8, 2, 31), (3, 5, 18, 6, 2, 32), (5, 4, 16, 5, 2, 33),
                                    (7, 3, 14, 5, 2, 34), (20, 3, 12, 4, 1, 35), (20, 4, 10, 3, 2, 36)]:
        alpha = alphabet_of(sigma)
        inst = pi.planted_instance_sigma(n, m, l, d, seed, alpha.encode())
        for q in [0] + list(range(1, n)):
            bf = o.sigma_bruteforce(inst.seqs, l, d, alpha, q=q)
            got = o.sigma_solve(inst.seqs, l, d, alpha, q=q, threads=2)
            assert np.array_equal(got, bf), (sigma, n, m, l, d, q)
            assert inst.motif.decode() in as_strings(got)
        seqs = random_over(rng, alpha, (n, m))
        assert np.array_equal(o.sigma_solve(seqs, l, d, alpha, threads=2), o.sigma_bruteforce(seqs, l, d, alpha))


def check_sigma_matches_dna(o) -> None:
    # over A, C, G, T the general search is the DNA search
    for (n, m, l, d, seed) in [(8, 60, 9, 2, 41), (6, 40, 10, 3, 42)]:
        inst = pi.planted_instance(n, m, l, d, seed)
        want = [o.decode(int(k), l) for k in o.solve(inst.seqs, l, d, threads=2)]
        assert as_strings(o.sigma_solve(inst.seqs, l, d, ACGT, threads=2)) == want
    inst = pi.planted_instance(6, 40, 8, 2, 43)
    wq = [o.decode(int(k), 8) for k in o.solve_quorum(inst.seqs, 8, 2, 4, threads=2)]
    assert as_strings(o.sigma_solve(inst.seqs, 8, 2, ACGT, q=4, threads=2)) == wq


def check_sigma_relabelling(o) -> None:
    # renaming the letters renames the motifs; the output order follows the alphabet given
    inst = pi.planted_instance_sigma(5, 30, 6, 2, 51, PROTEIN.encode())
    base = as_strings(o.sigma_solve(inst.seqs, 6, 2, PROTEIN, threads=2))
    assert inst.motif.decode() in base
    perm = np.random.default_rng(52).permutation(20)
    alt = "".join("abcdefghijklmnopqrst"[i] for i in perm)        # letter PROTEIN[k] -> alt[k]
    table = bytes.maketrans(PROTEIN.encode(), alt.encode())
    seqs2 = np.frombuffer(inst.seqs.tobytes().translate(table), dtype=np.uint8).reshape(inst.seqs.shape)
    got = as_strings(o.sigma_solve(seqs2, 6, 2, alt, threads=2))
    assert sorted(got) == sorted(s.translate(str.maketrans(PROTEIN, alt)) for s in base)
    key = [[alt.index(ch) for ch in s] for s in got]
    assert key == sorted(key)                                      # index order of the given alphabet
    assert len(set(got)) == len(got)


def check_sigma_special_cases(o) -> None:
    # d = 0: the l-mers present in every sequence
    inst = pi.planted_instance_sigma(4, 40, 3, 0, 61, b"ACD")
    sets = [lmers(bytes(row), 3) for row in inst.seqs]
    want = sorted(set.intersection(*sets), key=lambda s: ["ACD".index(c) for c in s])
    assert as_strings(o.sigma_solve(inst.seqs, 3, 0, "ACD", threads=1)) == want
    # n = 1, m = l: exactly the sphere B(x, d)
    x = "MKVLA"
    got = as_strings(o.sigma_solve(np.frombuffer(x.encode(), np.uint8).reshape(1, 5), 5, 2, PROTEIN, threads=1))
    assert len(got) == n_ball_sigma(5, 2, 20)
    assert all(py_hamming(x, s) <= 2 for s in got)
    # protein instances: the planted motif is found and every answer is a motif
    for (l, d, seed) in [(7, 2, 62), (8, 3, 63)]:
        inst = pi.planted_instance_sigma(10, 50, l, d, seed)
        got = as_strings(o.sigma_solve(inst.seqs, l, d, PROTEIN))
        assert inst.motif.decode() in got
        for s in got:
            assert o.is_motif(s, inst.seqs, d)


ALL_PINS = [check_compression_example, check_distance_definitions, check_neighbourhood_counts,
            check_neighbourhood_members, check_pair_intersections, check_bruteforce_agreement,
            check_planted_motif_found, check_special_cases, check_invariants, check_quorum, check_packed_solver,
            check_sigma_compression, check_sigma_neighbourhood_counts, check_sigma_bruteforce,
            check_sigma_matches_dna, check_sigma_relabelling, check_sigma_special_cases]
