"""Seeded synthetic planted-motif instances (the FM model: fixed number of mutations).

This module is shared by the oracle's tests and by the GPU library's tests and
benchmark, so it deliberately contains none of the motif-search method: only a
counter-based random number generator and the planting recipe.

Random numbers: SplitMix64 used as a counter-based generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): draw k
of stream s is mix64(s + (k + 1) * 0x9E3779B97F4A7C15), where mix64 is the
SplitMix64 output function. Bounded integers use the multiply-shift map
((u >> 32) * R) >> 32.

Instance recipe (the paper's FM data model, Sec. "Experimental Results"):
  * n sequences of length m, bases i.i.d. uniform over {A, C, G, T};
  * one uniform random l-mer motif;
  * per sequence: a uniform start position in [0, m - l], exactly d distinct
    positions of the copy picked by a partial Fisher-Yates shuffle, each
    changed to one of the three other bases uniformly, the copy overwriting
    the sequence there.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ALPHABET = b"ACGT"
_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(stream: int, counters) -> np.ndarray:
    """Draws ``counters`` (array of non-negative ints) of SplitMix64 stream ``stream``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(stream & _M64) + (c + np.uint64(1)) * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def bounded(u: np.ndarray, r) -> np.ndarray:
    """Maps 64-bit draws to integers in [0, r) by multiply-shift on the top 32 bits."""
    return ((np.asarray(u, dtype=np.uint64) >> np.uint64(32)) * np.asarray(r, dtype=np.uint64)) >> np.uint64(32)


def unit_float(u: np.ndarray) -> np.ndarray:
    """Maps 64-bit draws to floats in [0, 1) using the top 53 bits."""
    return (np.asarray(u, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


@dataclass
class Instance:
    seqs: np.ndarray      # (n, m) uint8, ASCII 'A','C','G','T'
    motif: bytes          # the planted l-mer
    positions: np.ndarray # (n,) start of each planted copy
    l: int
    d: int
    seed: int

    @property
    def n(self) -> int:
        return int(self.seqs.shape[0])

    @property
    def m(self) -> int:
        return int(self.seqs.shape[1])


def planted_instance(n: int, m: int, l: int, d: int, seed: int) -> Instance:
    """One FM-model instance: n random sequences of length m with an (l, d) motif planted once in each."""
    if not (1 <= l <= m) or not (0 <= d <= l) or n < 1:
        raise ValueError("need n >= 1, 1 <= l <= m, 0 <= d <= l")
    nm = n * m
    u = splitmix64(seed, np.arange(nm + l + n * (1 + 2 * d), dtype=np.uint64))
    alpha = np.frombuffer(ALPHABET, dtype=np.uint8)
    codes = (u[:nm] >> np.uint64(62)).astype(np.int64).reshape(n, m)
    motif = (u[nm:nm + l] >> np.uint64(62)).astype(np.int64)
    positions = np.zeros(n, dtype=np.int64)
    for i in range(n):
        c0 = nm + l + i * (1 + 2 * d)
        pos = int(bounded(u[c0], m - l + 1))
        copy = motif.copy()
        order = list(range(l))
        for k in range(d):
            j = k + int(bounded(u[c0 + 1 + k], l - k))
            order[k], order[j] = order[j], order[k]
            p = order[k]
            copy[p] = (copy[p] + 1 + int(bounded(u[c0 + 1 + d + k], 3))) % 4
        codes[i, pos:pos + l] = copy
        positions[i] = pos
    seqs = alpha[codes].astype(np.uint8)
    return Instance(seqs=np.ascontiguousarray(seqs), motif=bytes(alpha[motif]), positions=positions,
                    l=l, d=d, seed=seed)


#: the twenty amino acids, one-letter codes in alphabetical order
PROTEIN = b"ACDEFGHIKLMNPQRSTVWY"


def planted_instance_sigma(n: int, m: int, l: int, d: int, seed: int, alphabet: bytes = PROTEIN) -> Instance:
    """The FM recipe over a general alphabet of sigma letters: letters i.i.d. uniform, one uniform
    motif, per string one copy with exactly d distinct positions each changed to one of the
    sigma - 1 other letters uniformly."""
    alphabet = bytes(alphabet)
    sigma = len(alphabet)
    if sigma < 2 or len(set(alphabet)) != sigma:
        raise ValueError("need at least two distinct letters")
    if not (1 <= l <= m) or not (0 <= d <= l) or n < 1:
        raise ValueError("need n >= 1, 1 <= l <= m, 0 <= d <= l")
    nm = n * m
    u = splitmix64(seed, np.arange(nm + l + n * (1 + 2 * d), dtype=np.uint64))
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    codes = bounded(u[:nm], sigma).astype(np.int64).reshape(n, m)
    motif = bounded(u[nm:nm + l], sigma).astype(np.int64)
    positions = np.zeros(n, dtype=np.int64)
    for i in range(n):
        c0 = nm + l + i * (1 + 2 * d)
        pos = int(bounded(u[c0], m - l + 1))
        copy = motif.copy()
        order = list(range(l))
        for k in range(d):
            j = k + int(bounded(u[c0 + 1 + k], l - k))
            order[k], order[j] = order[j], order[k]
            p = order[k]
            copy[p] = (copy[p] + 1 + int(bounded(u[c0 + 1 + d + k], sigma - 1))) % sigma
        codes[i, pos:pos + l] = copy
        positions[i] = pos
    seqs = alpha[codes].astype(np.uint8)
    return Instance(seqs=np.ascontiguousarray(seqs), motif=bytes(alpha[motif]), positions=positions,
                    l=l, d=d, seed=seed)


def random_sequences(n: int, m: int, seed: int) -> np.ndarray:
    """n i.i.d. uniform DNA sequences of length m (no planted motif)."""
    u = splitmix64(seed, np.arange(n * m, dtype=np.uint64))
    alpha = np.frombuffer(ALPHABET, dtype=np.uint8)
    return np.ascontiguousarray(alpha[(u >> np.uint64(62)).astype(np.int64)].reshape(n, m))


# --- the benchmark workloads ------------------------------------------------

#: plain single-instance configurations: (l, d) with n = 20, m = 600
PLAIN_LD = [(9, 2), (15, 4), (17, 5), (19, 6)]

#: protein (20-letter) single-instance configurations: (l, d) with n = 20, m = 600
PROTEIN_LD = [(9, 3), (9, 4)]


def plain_instance(l: int, d: int, seed: int = 1, n: int = 20, m: int = 600) -> Instance:
    return planted_instance(n, m, l, d, seed)


def batch_instances(count: int = 256, master_seed: int = 2024,
                    ld_choices=((11, 3), (13, 4), (15, 4)),
                    n_range=(10, 30), m_range=(300, 1000)) -> list[Instance]:
    """The batched workload: (l, d), n and m drawn uniformly per instance."""
    u = splitmix64(master_seed, np.arange(4 * count, dtype=np.uint64)).reshape(count, 4)
    out = []
    for k in range(count):
        l, d = ld_choices[int(bounded(u[k, 0], len(ld_choices)))]
        n = n_range[0] + int(bounded(u[k, 1], n_range[1] - n_range[0] + 1))
        m = m_range[0] + int(bounded(u[k, 2], m_range[1] - m_range[0] + 1))
        out.append(planted_instance(n, m, l, d, int(u[k, 3])))
    return out


def serve_requests(count: int = 10000, rate_per_s: float = 200.0, master_seed: int = 7,
                   ld_choices=((13, 4), (15, 4), (17, 5)), n: int = 20,
                   m_range=(200, 1200)):
    """The served workload: Poisson arrivals; yields (arrival_time_s, Instance) lazily."""
    u = splitmix64(master_seed, np.arange(4 * count, dtype=np.uint64)).reshape(count, 4)
    gaps = -np.log1p(-unit_float(u[:, 0])) / rate_per_s
    t = np.cumsum(gaps)
    for k in range(count):
        l, d = ld_choices[int(bounded(u[k, 1], len(ld_choices)))]
        m = m_range[0] + int(bounded(u[k, 2], m_range[1] - m_range[0] + 1))
        yield float(t[k]), planted_instance(n, m, l, d, int(u[k, 3]))
