"""The three-string feasibility theorem of TraverStringRef (the paper's "Feasibility
Check without Precomputed Table"), read with 2·|R5| in its last inequality, pinned by
brute force over every string of small length.

B(a, da) ∩ B(b, db) ∩ B(c, dc) is non-empty iff da, db, dc >= 0, the three pairwise
sums cover the pairwise distances, and da + db + dc >= |R2| + |R3| + |R4| + 2·|R5|
(R2: a = b != c, R3: c = a != b, R4: b = c != a, R5: all three differ). The paper prints
the last term as |R5|; a position where all three differ costs at least 2 to any
string, and the brute force below shows that |R5| alone admits empty intersections.

In bit-plane form, with D = mism(a, b), Dw = mism(a, c), E = mism(b, c):
|R2| + |R3| + |R4| + 2|R5| = popc(Dw & E) + popc(D), so for da = db = dc = d the last
inequality is popc(Dw & E) <= 3d - popc(D), the root bound the pair form applies to
every occurrence c of a seed pair (a, b).
"""
import itertools
import random

ALPHA = "ACGT"


def hamming(u, v):
    return sum(1 for p, q in zip(u, v) if p != q)


def brute_nonempty(a, b, c, da, db, dc):
    for m in itertools.product(ALPHA, repeat=len(a)):
        if hamming(m, a) <= da and hamming(m, b) <= db and hamming(m, c) <= dc:
            return True
    return False


def classes(a, b, c):
    r2 = sum(1 for p, q, s in zip(a, b, c) if p == q != s)
    r3 = sum(1 for p, q, s in zip(a, b, c) if s == p != q)
    r4 = sum(1 for p, q, s in zip(a, b, c) if q == s != p)
    r5 = sum(1 for p, q, s in zip(a, b, c) if p != q and q != s and s != p)
    return r2, r3, r4, r5


def theorem(a, b, c, da, db, dc, r5_weight=2):
    r2, r3, r4, r5 = classes(a, b, c)
    return (min(da, db, dc) >= 0 and da + db >= hamming(a, b) and db + dc >= hamming(b, c)
            and dc + da >= hamming(c, a) and da + db + dc >= r2 + r3 + r4 + r5_weight * r5)


def _cases(l, count, seed):
    rng = random.Random(seed)
    for _ in range(count):
        a, b, c = ("".join(rng.choice(ALPHA) for _ in range(l)) for _ in range(3))
        yield a, b, c, rng.randint(0, l), rng.randint(0, l), rng.randint(0, l)


def test_theorem_matches_brute_force():
    for l in (1, 2, 3, 4, 5):
        for a, b, c, da, db, dc in _cases(l, 400, 11 + l):
            assert theorem(a, b, c, da, db, dc) == brute_nonempty(a, b, c, da, db, dc), (a, b, c, da, db, dc)


def test_printed_single_r5_term_is_not_sufficient():
    # all three letters differ at both positions: the printed |R5| term allows radii
    # whose intersection is empty
    a, b, c = "AA", "CC", "GG"
    assert theorem(a, b, c, 1, 1, 1, r5_weight=1)
    assert not brute_nonempty(a, b, c, 1, 1, 1)
    assert not theorem(a, b, c, 1, 1, 1)


def planes(s):
    hi = lo = 0
    for k, ch in enumerate(s):
        code = ALPHA.index(ch)
        hi |= (code >> 1) << k
        lo |= (code & 1) << k
    return hi, lo


def test_bit_plane_form_of_the_last_inequality():
    for l in (3, 6, 9):
        for a, b, c, _, _, _ in _cases(l, 300, 5 + l):
            (ah, al), (bh, bl), (ch, cl) = planes(a), planes(b), planes(c)
            D = (ah ^ bh) | (al ^ bl)
            Dw = (ah ^ ch) | (al ^ cl)
            E = (bh ^ ch) | (bl ^ cl)
            r2, r3, r4, r5 = classes(a, b, c)
            assert r2 + r3 + r4 + 2 * r5 == bin(Dw & E).count("1") + bin(D).count("1")


# ---- the same test below a tree node (the verification kernel's triple_rows option)
#
# A node P of seed x holds the strings c with c = x outside P and c != x on P.
# For occurrences u, w let t_u = popc(mism(x, u) ^ P) and F = the positions of
# P where x, u and w are three different letters; some string of the node is
# within d of both u and w iff t_u <= d, t_w <= d and t_u + t_w + F <= 2d.


def node_strings(x, P):
    choices = [[ch for ch in ALPHA if ch != x[p]] if p in P else [x[p]] for p in range(len(x))]
    for t in itertools.product(*choices):
        yield "".join(t)


def node_pair_feasible(x, u, w, P, d):
    Du = {p for p in range(len(x)) if u[p] != x[p]}
    Dw = {p for p in range(len(x)) if w[p] != x[p]}
    tu = len(Du ^ P)
    tw = len(Dw ^ P)
    F = sum(1 for p in P if u[p] != x[p] and w[p] != x[p] and u[p] != w[p])
    return tu <= d and tw <= d and tu + tw + F <= 2 * d


def test_node_pair_test_matches_brute_force():
    rng = random.Random(2403)
    for l in (2, 3, 4, 5, 6):
        for _ in range(300):
            x, u, w = ("".join(rng.choice(ALPHA) for _ in range(l)) for _ in range(3))
            P = {p for p in range(l) if rng.random() < 0.5}
            d = rng.randint(0, l)
            brute = any(hamming(c, u) <= d and hamming(c, w) <= d for c in node_strings(x, P))
            assert node_pair_feasible(x, u, w, P, d) == brute, (x, u, w, sorted(P), d)


def test_node_pair_test_in_bit_planes():
    # the kernel's form: Du = mism(x, u), t_u = popc(Du ^ P), F = popc(Du & Dw & mism(u, w) & P)
    rng = random.Random(7)
    for l in (5, 9, 15):
        for _ in range(300):
            x, u, w = ("".join(rng.choice(ALPHA) for _ in range(l)) for _ in range(3))
            P = {p for p in range(l) if rng.random() < 0.4}
            Pm = sum(1 << p for p in P)
            (xh, xl), (uh, ul), (wh, wl) = planes(x), planes(u), planes(w)
            Du = (xh ^ uh) | (xl ^ ul)
            Dw = (xh ^ wh) | (xl ^ wl)
            Euw = (uh ^ wh) | (ul ^ wl)
            F = bin(Du & Dw & Euw & Pm).count("1")
            assert F == sum(1 for p in P if len({x[p], u[p], w[p]}) == 3)
            assert bin(Du ^ Pm).count("1") == len({p for p in range(l) if u[p] != x[p]} ^ P)
