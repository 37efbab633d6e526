"""The CPU oracle against the paper's worked example, closed forms, brute force and invariants."""
import numpy as np
import pytest

import planted_inputs as pi
import oracle_pins as pins


@pytest.mark.parametrize("check", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(oracle_, check):
    check(oracle_)


def test_closed_form_values():
    # Values of the sphere size n_B(l, d) used elsewhere in the build notes.
    assert [pins.n_ball(l, d) for (l, d) in [(9, 2), (11, 3), (13, 4), (15, 4), (15, 5), (17, 5), (19, 6)]] == \
        [352, 4984, 66379, 123841, 853570, 1716100, 22946548]
    # the pair-class count reduces to the sphere size at D = 0 and to C(2d, d) at D = 2d
    for (l, d) in [(9, 2), (15, 4), (19, 6)]:
        assert pins.pair_ball_size(l, d, 0) == pins.n_ball(l, d)
        assert pins.pair_ball_size(l, d, 2 * d) == __import__("math").comb(2 * d, d)


def test_pair_size_19_6_by_distance():
    want = [22946548, 9413392, 6406024, 3693496, 2268436, 1297102, 720214, 370230, 174846,
            72576, 25116, 6468, 924]
    assert [pins.pair_ball_size(19, 6, D) for D in range(13)] == want


def test_oracle_pair_walk_19_6(oracle_):
    # one full B(x, 6) walk at l = 19 with r at distance 12: only C(12, 6) strings survive
    x = "ACGTACGTACGTACGTACG"
    r = list(x)
    for p in range(12):
        r[p] = "ACGT"[("ACGT".index(r[p]) + 2) % 4]
    assert oracle_.pair_intersection_size(x, "".join(r), 6) == 924


def test_plain_9_2_full_size(oracle_):
    # the (9, 2) plain configuration at its full size (n = 20, m = 600)
    for seed in (1, 2):
        inst = pi.plain_instance(9, 2, seed=seed)
        got = oracle_.solve(inst.seqs, 9, 2)
        assert pins.py_key(inst.motif.decode()) in set(int(k) for k in got)
        for k in got:
            assert oracle_.is_motif(oracle_.decode(int(k), 9), inst.seqs, 2)
        assert np.array_equal(got, oracle_.solve_pairs(inst.seqs, 9, 2))


def test_invalid_input_rejected(oracle_):
    seqs = pi.random_sequences(3, 20, 1).copy()
    seqs[1, 4] = ord("N")
    with pytest.raises(ValueError):
        oracle_.solve(seqs, 5, 1)
    ok = pi.random_sequences(3, 20, 1)
    for (l, d) in [(0, 0), (21, 1), (5, 5), (5, -1), (33, 2)]:
        with pytest.raises(ValueError):
            oracle_.solve(ok, l, d)
