"""The general-alphabet node search, compiled for the host from the kernel's own source,
against the oracle on small instances, with no GPU:

* tests/host/sigma_search_host.cu runs it with a one-thread group (rows built on the host
  in the kernel's layout): the search logic (node bound, letter classes, depth-first
  prefixes, pivot rows, witness rows), and the same search with the row lists shrunk
  depth by depth (the list form the kernel takes when a node's lists fit, with a small
  buffer too, so that nodes fall back to the form without lists);
* tests/host/sigma_search_lockstep.cu runs it with 32 host threads per node whose votes,
  broadcasts and sums go through barriers, sharing the per-warp state and witness rows:
  the lane-parallel form the GPU warp executes (row scans split over 32 lanes, one lane
  reserving output slots, every lane writing the shared state)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import planted_inputs as pi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "sigma_search_host.cu")


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


@pytest.fixture(scope="module")
def search(tmp_path_factory):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("sigma") / "sigma_search_host")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-diag-suppress", "550", "-I", os.path.join(ROOT, "include"), SRC, "-o", exe],
                   check=True, capture_output=True)

    def run(seqs, l, d, alphabet, q=0, lists=0, packed=0):
        n, m = seqs.shape
        inp = f"{alphabet} {n} {m} {l} {d} {q}\n" + "\n".join(bytes(r).decode() for r in seqs) + "\n"
        r = subprocess.run([exe, str(lists), str(packed)], input=inp, capture_output=True, text=True, check=True)
        return r.stdout.split()
    run.exe = exe
    return run


def test_node_ranks_are_a_bijection_onto_the_subsets(search):
    # rank r -> position subset: every subset of at most d of the l positions exactly once,
    # sizes in increasing order (the search visits the tree's nodes through these ranks)
    import itertools
    for l, d in [(1, 0), (5, 5), (9, 4), (12, 3), (32, 2)]:
        r = subprocess.run([search.exe], input=f"unrank {l} {d}\n", capture_output=True, text=True, check=True)
        got = [int(v) for v in r.stdout.split()]
        want = {sum(1 << p for p in c) for k in range(d + 1) for c in itertools.combinations(range(l), k)}
        assert len(got) == len(want) and set(got) == want, (l, d)
        sizes = [bin(v).count("1") for v in got]
        assert sizes == sorted(sizes)


def alphabet_of(sigma: int) -> str:
    return "".join(reversed("ACDEFGHIKLMNPQRSTVWYBJOUXZ0123456789"[:sigma]))


CASES = [
    # sigma, n, m, l, d, q, seed
    (2, 6, 40, 10, 2, 0, 1), (3, 5, 30, 7, 3, 4, 4), (4, 8, 60, 9, 2, 0, 5), (7, 5, 40, 6, 2, 3, 7),
    (17, 5, 30, 5, 2, 0, 9), (20, 6, 50, 6, 3, 0, 11), (20, 5, 40, 6, 3, 3, 12), (32, 5, 30, 5, 2, 4, 15),
    (20, 1, 9, 5, 2, 0, 16), (20, 6, 30, 4, 0, 0, 17), (5, 4, 6, 6, 3, 0, 18), (20, 7, 33, 32, 1, 0, 19),
    (4, 5, 40, 32, 2, 0, 20),   # b l = 64: the packed word exactly full
]


# packed = 1: rows in the kernel's packed layout (all planes in one 64-bit word) wherever
# 2 <= b and b l <= 64, i.e. every case here but sigma = 2 and (20 letters, l = 32)
@pytest.mark.parametrize("lists,packed", [(0, 0), (4096, 0), (24, 0), (0, 1), (4096, 1), (24, 1)])
@pytest.mark.parametrize("sigma,n,m,l,d,q,seed", CASES)
def test_host_search_matches_the_oracle(search, oracle_, sigma, n, m, l, d, q, seed, lists, packed):
    alpha = alphabet_of(sigma)
    inst = pi.planted_instance_sigma(n, m, l, d, seed, alpha.encode())
    want = [bytes(r).decode() for r in oracle_.sigma_solve(inst.seqs, l, d, alpha, q=q, cap=1 << 22)]
    assert search(inst.seqs, l, d, alpha, q, lists, packed) == want


def test_host_search_over_acgt_matches_the_dna_oracle(search, oracle_):
    inst = pi.planted_instance(10, 120, 10, 3, 21)
    want = [oracle_.decode(int(k), 10) for k in oracle_.solve(inst.seqs, 10, 3)]
    assert search(inst.seqs, 10, 3, "ACGT") == want


def test_host_search_on_random_backgrounds(search, oracle_):
    rng = np.random.default_rng(5)
    for sigma, n, m, l, d in [(20, 6, 40, 6, 3), (3, 8, 60, 9, 3), (2, 10, 50, 12, 3)]:
        alpha = alphabet_of(sigma)
        letters = np.frombuffer(alpha.encode(), np.uint8)
        seqs = letters[rng.integers(0, sigma, size=(n, m))].astype(np.uint8)
        for q in (0, n - 1):
            want = [bytes(r).decode() for r in oracle_.sigma_solve(seqs, l, d, alpha, q=q, cap=1 << 22)]
            assert search(seqs, l, d, alpha, q) == want, (sigma, n, m, l, d, q)
            assert search(seqs, l, d, alpha, q, 4096) == want, (sigma, n, m, l, d, q, "lists")
            assert search(seqs, l, d, alpha, q, 4096, 1) == want, (sigma, n, m, l, d, q, "lists, packed")


@pytest.fixture(scope="module")
def lockstep(tmp_path_factory):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("sigma_lockstep") / "sigma_search_lockstep")
    subprocess.run([nvcc, "-O2", "-std=c++20", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-diag-suppress", "550,177", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "host", "sigma_search_lockstep.cu"), "-o", exe],
                   check=True, capture_output=True)

    def run(seqs, l, d, alphabet, q=0, lists=0, packed=0):
        n, m = seqs.shape
        inp = f"{alphabet} {n} {m} {l} {d} {q}\n" + "\n".join(bytes(r).decode() for r in seqs) + "\n"
        r = subprocess.run([exe, str(lists), str(packed)], input=inp, capture_output=True, text=True, check=True,
                           timeout=300)
        return r.stdout.split()
    return run


# tiny cases (every collective is a barrier of 32 host threads): protein and DNA instances that
# take the pivot form, a quorum and n = 1 that take the plain depth-first form
LOCKSTEP_CASES = [(20, 4, 20, 5, 2, 0, 31), (3, 4, 16, 6, 2, 3, 33), (20, 1, 7, 4, 2, 0, 34),
                  (4, 6, 30, 8, 2, 0, 35), (4, 8, 60, 9, 2, 0, 5)]


@pytest.mark.parametrize("lists,packed", [(0, 0), (4096, 0), (4096, 1)])
@pytest.mark.parametrize("sigma,n,m,l,d,q,seed", LOCKSTEP_CASES)
def test_lane_parallel_search_matches_the_oracle(lockstep, oracle_, sigma, n, m, l, d, q, seed, lists, packed):
    alpha = alphabet_of(sigma)
    inst = pi.planted_instance_sigma(n, m, l, d, seed, alpha.encode())
    want = [bytes(r).decode() for r in oracle_.sigma_solve(inst.seqs, l, d, alpha, q=q, cap=1 << 22)]
    assert lockstep(inst.seqs, l, d, alpha, q, lists, packed) == want
