"""Helpers shared by the GPU parity tests (no method arithmetic of the library is reused here)."""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}


def seq_codes(seqs: np.ndarray) -> np.ndarray:
    lut = np.full(256, 255, dtype=np.uint8)
    for k, v in CODE.items():
        lut[k] = v
    return lut[np.asarray(seqs, dtype=np.uint8)]


def key_digits(keys: np.ndarray, l: int) -> np.ndarray:
    """(len(keys), l) array of base codes of each motif key (position 0 = most significant)."""
    keys = np.asarray(keys, dtype=np.uint64)
    shifts = np.array([2 * (l - 1 - p) for p in range(l)], dtype=np.uint64)
    return ((keys[:, None] >> shifts[None, :]) & np.uint64(3)).astype(np.uint8)


def keys_within(keys: np.ndarray, x_codes: np.ndarray, l: int, d: int) -> np.ndarray:
    """The keys whose string is within Hamming distance d of the l-mer x (given as codes)."""
    if len(keys) == 0:
        return np.asarray(keys, dtype=np.uint64)
    dig = key_digits(keys, l)
    dist = (dig != x_codes[None, :]).sum(axis=1)
    return np.asarray(keys, dtype=np.uint64)[dist <= d]


def oracle_per_seed(o, seqs: np.ndarray, l: int, d: int, seeds, workers: int | None = None) -> dict:
    """{seed j: oracle motifs inside B(s_1[j..j+l-1], d)}, seeds computed in parallel threads."""
    workers = workers or max(1, (os.cpu_count() or 2))

    def one(j):
        return j, o.solve_seeds(seqs, l, d, j, j + 1, threads=1)

    with ThreadPoolExecutor(workers) as ex:
        return dict(ex.map(one, list(seeds)))


def py_key(s: str) -> int:
    k = 0
    for ch in s:
        k = 4 * k + "ACGT".index(ch)
    return k
