"""CPU oracle for exact planted (l,d)-motif search -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The GPU library never does, and this
package imports nothing from it: the two share no code. The arithmetic lives
in ``pms_oracle.c`` (plain C, compiled here with gcc on first use); this file
only marshals arguments.

What it computes is the definition itself (Definitions 3-5 of the paper with
q = n): the set of l-mers M over {A,C,G,T} such that every input sequence has
a window within Hamming distance d of M. The candidate set is restricted by
Observation 3.1 (every motif lies in B(x, d) for some l-mer x of s_1), which
is exact for q = n. Variants: the pair form of Observation 3.3, and the
pattern-driven brute force over all 4^l strings for tiny l. The same
definitions over a general alphabet (qPMS-Sigma: sigma distinct letters,
ceil(log2 sigma) bit-plane groups) are the ``sigma_*`` methods.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pms_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpms_oracle.so")
_lock = threading.Lock()
_lib = None

ALPHABET = "ACGT"


def build(force: bool = False, extra_flags: tuple = (), out_path: str | None = None) -> str:
    """Compiles pms_oracle.c with gcc into a shared library and returns its path."""
    out = out_path or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", *extra_flags, _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _declare(lib):
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    c_int, c_long = ctypes.c_int, ctypes.c_long
    sig = {
        "oracle_hamming": (c_int, [u8p, u8p, c_int]),
        "oracle_distance_to_string": (c_int, [u8p, c_int, u8p, c_int]),
        "oracle_is_motif": (c_int, [u8p, c_int, c_int, u8p, c_int, c_int]),
        "oracle_compress": (c_int, [u8p, c_int, u32p]),
        "oracle_compressed_distance": (c_int, [u32p, u32p, c_int]),
        "oracle_key": (ctypes.c_uint64, [u8p, c_int]),
        "oracle_decode": (None, [ctypes.c_uint64, c_int, u8p]),
        "oracle_neighbourhood": (c_long, [u8p, c_int, c_int, u64p, c_long]),
        "oracle_neighbourhood_visits": (c_long, [u8p, c_int, c_int]),
        "oracle_pair_intersection_size": (c_long, [u8p, u8p, c_int, c_int]),
        "oracle_solve": (c_long, [u8p, c_int, c_int, c_int, c_int, c_int, u64p, c_long]),
        "oracle_solve_seeds": (c_long, [u8p, c_int, c_int, c_int, c_int, c_long, c_long, c_int, u64p, c_long]),
        "oracle_solve_pairs": (c_long, [u8p, c_int, c_int, c_int, c_int, c_int, u64p, c_long]),
        "oracle_solve_pairs_seeds": (c_long, [u8p, c_int, c_int, c_int, c_int, c_long, c_long, c_int, u64p,
                                               c_long]),
        "oracle_solve_packed": (c_long, [u8p, c_int, c_int, c_int, c_int, c_long, c_long, c_int, u64p, c_long]),
        "oracle_bruteforce": (c_long, [u8p, c_int, c_int, c_int, c_int, u64p, c_long]),
        "oracle_is_qmotif": (c_int, [u8p, c_int, c_int, c_int, u8p, c_int, c_int]),
        "oracle_solve_quorum": (c_long, [u8p, c_int, c_int, c_int, c_int, c_int, c_int, u64p, c_long]),
        "oracle_solve_quorum_seeds": (c_long, [u8p, c_int, c_int, c_int, c_int, c_int, c_long, c_long, c_int, u64p,
                                                c_long]),
        "oracle_bruteforce_quorum": (c_long, [u8p, c_int, c_int, c_int, c_int, c_int, u64p, c_long]),
        "oracle_sigma_groups": (c_int, [c_int]),
        "oracle_sigma_compress": (c_int, [u8p, c_int, u8p, c_int, u32p]),
        "oracle_sigma_compressed_distance": (c_int, [u32p, u32p, c_int, c_int]),
        "oracle_sigma_neighbourhood_visits": (c_long, [u8p, c_int, u8p, c_int, c_int]),
        "oracle_sigma_solve": (c_long, [u8p, c_int, u8p, c_int, c_int, c_int, c_int, c_int, c_int, u8p, c_long]),
        "oracle_sigma_solve_seeds": (c_long, [u8p, c_int, u8p, c_int, c_int, c_int, c_int, c_int, c_long, c_long,
                                               c_int, u8p, c_long]),
        "oracle_sigma_bruteforce": (c_long, [u8p, c_int, u8p, c_int, c_int, c_int, c_int, c_int, u8p, c_long]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load(path: str | None = None):
    """Loads (building if needed) the oracle library. ``path`` loads an alternative build."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _u8(buf) -> tuple:
    """A contiguous uint8 copy of ``buf`` and a ctypes pointer to it (keep both alive)."""
    if isinstance(buf, np.ndarray):
        arr = np.ascontiguousarray(buf, dtype=np.uint8)
    else:
        arr = np.frombuffer(bytes(buf), dtype=np.uint8).copy()
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _bytes(s) -> bytes:
    return s.encode() if isinstance(s, str) else bytes(s)


class Oracle:
    """Thin wrapper over one loaded oracle library (the default build or a variant)."""

    def __init__(self, lib=None):
        self.lib = lib or load()

    # --- single l-mers ---
    def hamming(self, a, b) -> int:
        a, b = _bytes(a), _bytes(b)
        (aa, pa), (bb, pb) = _u8(a), _u8(b)
        return int(self.lib.oracle_hamming(pa, pb, len(a)))

    def distance_to_string(self, x, s) -> int:
        x, s = _bytes(x), _bytes(s)
        (xa, px), (sa, ps) = _u8(x), _u8(s)
        return int(self.lib.oracle_distance_to_string(px, len(x), ps, len(s)))

    def compress(self, x) -> np.ndarray:
        x = _bytes(x)
        words = (len(x) + 31) // 32
        out = np.zeros(2 * words, dtype=np.uint32)
        xa, px = _u8(x)
        rc = self.lib.oracle_compress(px, len(x), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        if rc != 0:
            raise ValueError("not a DNA string")
        return out.reshape(2, words)

    def compressed_distance(self, a: np.ndarray, b: np.ndarray, l: int) -> int:
        a = np.ascontiguousarray(a, dtype=np.uint32).ravel()
        b = np.ascontiguousarray(b, dtype=np.uint32).ravel()
        p = ctypes.POINTER(ctypes.c_uint32)
        return int(self.lib.oracle_compressed_distance(a.ctypes.data_as(p), b.ctypes.data_as(p), l))

    def key(self, x) -> int:
        x = _bytes(x)
        xa, px = _u8(x)
        return int(self.lib.oracle_key(px, len(x)))

    def decode(self, key: int, l: int) -> str:
        out = np.zeros(l, dtype=np.uint8)
        self.lib.oracle_decode(ctypes.c_uint64(key), l, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        return out.tobytes().decode()

    # --- neighbourhoods ---
    def neighbourhood(self, x, d: int, cap: int = 1 << 22) -> np.ndarray:
        x = _bytes(x)
        xa, px = _u8(x)
        out = np.zeros(cap, dtype=np.uint64)
        n = self.lib.oracle_neighbourhood(px, len(x), d, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap)
        return self._result(n, out, cap)

    def neighbourhood_visits(self, x, d: int) -> int:
        x = _bytes(x)
        xa, px = _u8(x)
        return int(self.lib.oracle_neighbourhood_visits(px, len(x), d))

    def pair_intersection_size(self, x, r, d: int) -> int:
        x, r = _bytes(x), _bytes(r)
        (xa, px), (ra, pr) = _u8(x), _u8(r)
        return int(self.lib.oracle_pair_intersection_size(px, pr, len(x), d))

    # --- motif search ---
    def is_motif(self, M, seqs: np.ndarray, d: int) -> bool:
        M = _bytes(M)
        seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
        ma, pm = _u8(M)
        n, m = seqs.shape
        return bool(self.lib.oracle_is_motif(pm, len(M), d, seqs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), n, m))

    @staticmethod
    def _result(n: int, out: np.ndarray, cap: int) -> np.ndarray:
        if n == -1:
            raise ValueError("invalid input")
        if n == -2:
            raise MemoryError("oracle ran out of memory")
        if n > cap:
            raise OverflowError(f"{n} motifs exceed the output capacity {cap}")
        return out[:n].copy()

    def _solve(self, fn, seqs, l, d, *extra, cap=1 << 22):
        seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
        n, m = seqs.shape
        out = np.zeros(cap, dtype=np.uint64)
        p = seqs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        res = fn(p, n, m, l, d, *extra, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap)
        return self._result(res, out, cap)

    def solve(self, seqs, l: int, d: int, threads: int | None = None, cap: int = 1 << 22) -> np.ndarray:
        """All (l,d)-motifs as sorted unique keys."""
        return self._solve(self.lib.oracle_solve, seqs, l, d, threads or os.cpu_count() or 1, cap=cap)

    def solve_seeds(self, seqs, l: int, d: int, seed_lo: int, seed_hi: int, threads: int | None = None,
                    cap: int = 1 << 22) -> np.ndarray:
        """Motifs inside B(x, d) for seeds x = s_1[j..j+l-1], seed_lo <= j < seed_hi."""
        return self._solve(self.lib.oracle_solve_seeds, seqs, l, d, seed_lo, seed_hi,
                           threads or os.cpu_count() or 1, cap=cap)

    def solve_pairs(self, seqs, l: int, d: int, threads: int | None = None, cap: int = 1 << 22) -> np.ndarray:
        return self._solve(self.lib.oracle_solve_pairs, seqs, l, d, threads or os.cpu_count() or 1, cap=cap)

    def solve_pairs_seeds(self, seqs, l: int, d: int, seed_lo: int, seed_hi: int, threads: int | None = None,
                          cap: int = 1 << 22) -> np.ndarray:
        """solve_pairs restricted to the seeds x = s_1[j..j+l-1], seed_lo <= j < seed_hi."""
        return self._solve(self.lib.oracle_solve_pairs_seeds, seqs, l, d, seed_lo, seed_hi,
                           threads or os.cpu_count() or 1, cap=cap)

    def solve_packed(self, seqs, l: int, d: int, seed_lo: int = 0, seed_hi: int | None = None,
                     threads: int | None = None, cap: int = 1 << 22) -> np.ndarray:
        """The motifs inside B(x_j, d) for seeds j in [seed_lo, seed_hi) of s_1 (all of them by
        default, i.e. the whole motif set), with the motif test run on compressed l-mers."""
        W = np.asarray(seqs).shape[1] - l + 1
        hi = W if seed_hi is None else seed_hi
        return self._solve(self.lib.oracle_solve_packed, seqs, l, d, seed_lo, hi, threads or os.cpu_count() or 1,
                           cap=cap)

    def bruteforce(self, seqs, l: int, d: int, cap: int = 1 << 22) -> np.ndarray:
        return self._solve(self.lib.oracle_bruteforce, seqs, l, d, cap=cap)

    # --- quorum (qPMS) ---
    def is_qmotif(self, M, seqs: np.ndarray, d: int, q: int) -> bool:
        M = _bytes(M)
        seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
        ma, pm = _u8(M)
        n, m = seqs.shape
        return bool(self.lib.oracle_is_qmotif(pm, len(M), d, q, seqs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                              n, m))

    def solve_quorum(self, seqs, l: int, d: int, q: int, threads: int | None = None, cap: int = 1 << 22) -> np.ndarray:
        """All (l,d,q)-motifs as sorted unique keys."""
        return self._solve(self.lib.oracle_solve_quorum, seqs, l, d, q, threads or os.cpu_count() or 1, cap=cap)

    def solve_quorum_seeds(self, seqs, l: int, d: int, q: int, seed_lo: int, seed_hi: int,
                           threads: int | None = None, cap: int = 1 << 22) -> np.ndarray:
        """(l,d,q)-motifs inside B(x, d) for seeds [seed_lo, seed_hi) numbered over s_1, s_2, ..."""
        return self._solve(self.lib.oracle_solve_quorum_seeds, seqs, l, d, q, seed_lo, seed_hi,
                           threads or os.cpu_count() or 1, cap=cap)

    def bruteforce_quorum(self, seqs, l: int, d: int, q: int, cap: int = 1 << 22) -> np.ndarray:
        return self._solve(self.lib.oracle_bruteforce_quorum, seqs, l, d, q, cap=cap)

    def decode_all(self, keys, l: int) -> list[str]:
        return [self.decode(int(k), l) for k in keys]

    # --- general alphabets (qPMS-Sigma) ---
    def sigma_groups(self, sigma: int) -> int:
        return int(self.lib.oracle_sigma_groups(sigma))

    def sigma_compress(self, alphabet, x) -> np.ndarray:
        alphabet, x = _bytes(alphabet), _bytes(x)
        words = (len(x) + 31) // 32
        groups = self.sigma_groups(len(alphabet))
        out = np.zeros(groups * words, dtype=np.uint32)
        (aa, pa), (xa, px) = _u8(alphabet), _u8(x)
        rc = self.lib.oracle_sigma_compress(pa, len(alphabet), px, len(x),
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        if rc != 0:
            raise ValueError("invalid alphabet or letter")
        return out.reshape(groups, words)

    def sigma_compressed_distance(self, a: np.ndarray, b: np.ndarray, l: int) -> int:
        groups = np.asarray(a).shape[0]
        a = np.ascontiguousarray(a, dtype=np.uint32).ravel()
        b = np.ascontiguousarray(b, dtype=np.uint32).ravel()
        p = ctypes.POINTER(ctypes.c_uint32)
        return int(self.lib.oracle_sigma_compressed_distance(a.ctypes.data_as(p), b.ctypes.data_as(p), l, groups))

    def sigma_neighbourhood_visits(self, alphabet, x, d: int) -> int:
        alphabet, x = _bytes(alphabet), _bytes(x)
        (aa, pa), (xa, px) = _u8(alphabet), _u8(x)
        return int(self.lib.oracle_sigma_neighbourhood_visits(pa, len(alphabet), px, len(x), d))

    def _sigma(self, fn, alphabet, seqs, l, d, q, *extra, cap):
        alphabet = _bytes(alphabet)
        seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
        n, m = seqs.shape
        out = np.zeros(cap * l, dtype=np.uint8)
        aa, pa = _u8(alphabet)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        res = fn(pa, len(alphabet), seqs.ctypes.data_as(u8p), n, m, l, d, q, *extra, out.ctypes.data_as(u8p), cap)
        if res == -1:
            raise ValueError("invalid input")
        if res == -2:
            raise MemoryError("oracle ran out of memory")
        if res > cap:
            raise OverflowError(f"{res} motifs exceed the output capacity {cap}")
        return out[: res * l].reshape(res, l).copy()

    def sigma_solve(self, seqs, l: int, d: int, alphabet, q: int = 0, threads: int | None = None,
                    cap: int = 1 << 20) -> np.ndarray:
        """All (l,d,q)-motifs over ``alphabet`` (q = 0: q = n) as an (count, l) uint8 array of letters,
        rows in lexicographic order of the alphabet's indices."""
        return self._sigma(self.lib.oracle_sigma_solve, alphabet, seqs, l, d, q, threads or os.cpu_count() or 1,
                           cap=cap)

    def sigma_solve_seeds(self, seqs, l: int, d: int, alphabet, seed_lo: int, seed_hi: int, q: int = 0,
                          threads: int | None = None, cap: int = 1 << 20) -> np.ndarray:
        """The motifs inside B(x, d) for seeds [seed_lo, seed_hi) numbered over s_1..s_{n-q+1}."""
        return self._sigma(self.lib.oracle_sigma_solve_seeds, alphabet, seqs, l, d, q, seed_lo, seed_hi,
                           threads or os.cpu_count() or 1, cap=cap)

    def sigma_bruteforce(self, seqs, l: int, d: int, alphabet, q: int = 0, cap: int = 1 << 20) -> np.ndarray:
        return self._sigma(self.lib.oracle_sigma_bruteforce, alphabet, seqs, l, d, q, cap=cap)
