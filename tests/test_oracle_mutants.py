"""Planted mistakes in copies of the CPU oracle must each be caught by at least one pin.

Each mutant is pms_oracle.c with one plausible slip (a dropped term, a wrong
bound, a wrong index), compiled here with gcc into a temporary library. The
pins of oracle_pins.py are then run against it; the test fails if every pin
still passes, i.e. if the pins could not tell that oracle from the real one.
"""
import os

import pytest

import oracle
import oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "pms_oracle.c")

MUTANTS = {
    # strict instead of non-strict distance test (Definition 5 says "no more than d")
    "strict_threshold": ("if (oracle_hamming(x, s + j, l) <= d)", "if (oracle_hamming(x, s + j, l) < d)"),
    # last window of each sequence dropped (index range of Definition 2)
    "last_window_dropped": ("for (int j = 0; j + l <= m; ++j)\n        if (oracle_hamming",
                            "for (int j = 0; j + l < m; ++j)\n        if (oracle_hamming"),
    # last sequence never checked
    "last_sequence_skipped": ("for (int i = 0; i < n; ++i)\n        if (!string_has_occurrence",
                              "for (int i = 0; i < n - 1; ++i)\n        if (!string_has_occurrence"),
    # tree children may reuse the parent's position: duplicates and depth errors
    "tree_position_reused": ("walk_tree(w, p + 1, depth + 1);", "walk_tree(w, p, depth + 1);"),
    # tree skips the position right after the last change: misses strings
    "tree_position_skipped": ("walk_tree(w, p + 1, depth + 1);", "walk_tree(w, p + 2, depth + 1);"),
    # tree stops one level early
    "tree_too_shallow": ("if (depth == w->d)\n        return;", "if (depth + 1 >= w->d)\n        return;"),
    # two letters' codes swapped (C <-> G)
    "codes_swapped": ("case 'C': return 1;\n    case 'G': return 2;", "case 'C': return 2;\n    case 'G': return 1;"),
    # compressed distance ignores group 1
    "group_dropped": ("for (int g = 0; g < 2; ++g)\n            acc |=", "for (int g = 0; g < 1; ++g)\n            acc |="),
    # pair variant uses d instead of 2d for the pair filter
    "pair_filter_tight": ("> 2 * j->d)", "> j->d)"),
    # quorum: seeds only from s_1 (Observation 3.1 needs s_1..s_{n-q+1})
    "quorum_seeds_first_only": ("(q > 0 ? (long)(n - q + 1) : 1L) * W", "1L * W"),
    # quorum test off by one
    "quorum_threshold": ("if (hits >= q)\n            return 1;", "if (hits > q)\n            return 1;"),
    # general alphabets: the last letter of the alphabet never substituted
    "sigma_last_letter_skipped": ("for (int b = 0; b < w->sigma; ++b) {\n                if (w->alphabet[b]",
                                  "for (int b = 0; b < w->sigma - 1; ++b) {\n                if (w->alphabet[b]"),
    # general alphabets: one bit-plane group too few when sigma is one above a power of two
    "sigma_groups_short": ("while ((1 << g) < sigma)", "while ((1 << g) < sigma - 1)"),
    # general alphabets: duplicates across seeds kept
    "sigma_duplicates_kept": ("if (u == 0 || memcmp(", "if (u >= 0 || memcmp("),
    # general alphabets: the sphere stops one level early
    "sigma_tree_too_shallow": ("if (depth < w->d) {", "if (depth + 1 < w->d) {"),
    # general alphabets: quorum seeds only from s_1
    "sigma_quorum_seeds_first_only": ("(long)(q > 0 ? n - q + 1 : 1) * W", "(long)1 * W"),
    # general alphabets: brute force skips the last letter at the last position
    "sigma_bruteforce_counter": ("while (k >= 0 && idx[k] == sigma - 1)", "while (k >= 0 && idx[k] == sigma - 2)"),
    # compressed motif test: strict threshold
    "packed_strict_threshold": ("(cand[1] ^ hi[j])) <= pk->d;", "(cand[1] ^ hi[j])) < pk->d;"),
    # compressed motif test: group 1 ignored
    "packed_group_dropped": ("__builtin_popcount((cand[0] ^ lo[j]) | (cand[1] ^ hi[j]))",
                             "__builtin_popcount(cand[0] ^ lo[j])"),
    # compressed motif test: the last window of each string dropped
    "packed_last_window_dropped": ("for (int j = 0; j < pk->W && !found; ++j)",
                                   "for (int j = 0; j < pk->W - 1 && !found; ++j)"),
    # compressed motif test: s_n never checked (the strings run s_2 .. s_{n-1}, s_1)
    "packed_string_skipped": ("const int i = t % pk->n;", "const int i = (t % pk->n == pk->n - 1) ? 0 : t % pk->n;"),
    # Hamming distance counts matches instead of mismatches at the first position
    "hamming_first_position": ("for (int k = 0; k < l; ++k)\n        if (a[k] != b[k])",
                               "for (int k = 1; k < l; ++k)\n        if (a[k] != b[k])"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / f"lib{name}.so"
    import subprocess
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", str(path), "-o", str(lib)], check=True)
    return oracle.Oracle(oracle.load(str(lib)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    o = _build_mutant(tmp_path, name, old, new)
    failures = []
    for check in pins.ALL_PINS:
        try:
            check(o)
        except (AssertionError, ValueError, OverflowError) as e:  # a pin fired
            failures.append(check.__name__)
    assert failures, f"no pin detects the planted mistake {name}"
