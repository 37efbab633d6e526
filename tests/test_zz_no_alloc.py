"""The allocation-free entry point against the regular device entry point.

pms_solve_device_noalloc exists for callers that may not allocate device
memory while running (their memory is pre-planned and handed out by their own
allocator, or cudaMalloc/cudaFree may block or synchronize at a bad time): it
takes every buffer from one fixed per-GPU array in the library. This test
calls it through the C ABI twice in a row on the same stream and compares each
result with pms_solve_device on the same input (motif sets are exact: equal
codes, equal counts). It is collected last so a failure here does not hide the
other GPU tests, and it works alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms

pytestmark = pytest.mark.gpu


def _reference(ctx, torch, seqs, l, d, cap):
    n, m = seqs.shape
    d_in = torch.from_numpy(seqs.copy()).cuda()
    out = torch.zeros(cap, dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    ctx.solve_device(d_in, n, m, l, d, out, cap, st)
    torch.cuda.synchronize()
    s = st.cpu().numpy().astype(np.uint32)
    return s, out[: int(s[1])].cpu().numpy().astype(np.uint64)


def _noalloc(lib, torch, stream, seqs, l, d, cap):
    n, m = seqs.shape
    d_in = torch.from_numpy(seqs.copy()).cuda()
    out = torch.zeros(cap, dtype=torch.int64, device="cuda")
    st = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = lib.pms_solve_device_noalloc(ctypes.c_void_p(d_in.data_ptr()), n, m, l, d, ctypes.c_void_p(out.data_ptr()),
                                      cap, ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == pms.PMS_OK, pms.ERROR_NAMES.get(rc, rc)
    stream.synchronize()
    s = st.cpu().numpy().astype(np.uint32)
    return s, out[: int(s[1])].cpu().numpy().astype(np.uint64)


def test_noalloc_matches_device_entry_point_twice():
    import torch
    lib = pms.load()
    stream = torch.cuda.Stream()
    ctx = pms.Context(0)
    ctx.set_stream(stream)
    cap = 4096
    cases = [pi.plain_instance(15, 4, seed=21), pi.planted_instance(12, 300, 11, 3, 22)]
    for inst in cases:
        with torch.cuda.stream(stream):
            want_st, want = _reference(ctx, torch, inst.seqs, inst.l, inst.d, cap)
            got_st, got = _noalloc(lib, torch, stream, inst.seqs, inst.l, inst.d, cap)
        assert got_st[2] == want_st[2] == 0
        assert got_st[1] == want_st[1]
        assert np.array_equal(got, want)
        assert len(got) >= 1
    ctx.close()


def test_noalloc_rejects_too_large():
    import torch
    lib = pms.load()
    d_in = torch.zeros(64 * 4096, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = lib.pms_solve_device_noalloc(ctypes.c_void_p(d_in.data_ptr()), 64, 4096, 20, 5, ctypes.c_void_p(out.data_ptr()),
                                      16, ctypes.c_void_p(st.data_ptr()), None)
    assert rc == pms.PMS_ESCRATCH


def test_noalloc_raw_limit_reported_without_overrun():
    # n = 1 and a loose (l, d): B(x, 3) over 31 seeds holds far more than the
    # 65536 raw codes the fixed array keeps; the status reports the overflow
    # (flag bit 1, the full raw count) and no code is written past `capacity`
    import torch
    lib = pms.load()
    seqs = pi.random_sequences(1, 40, 91)
    n, m, l, d = 1, 40, 10, 3
    cap, slack = 1000, 64
    d_in = torch.from_numpy(seqs.copy()).cuda()
    out = torch.full((cap + slack,), -7, dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    rc = lib.pms_solve_device_noalloc(ctypes.c_void_p(d_in.data_ptr()), n, m, l, d, ctypes.c_void_p(out.data_ptr()),
                                      cap, ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == pms.PMS_OK
    stream.synchronize()
    s = st.cpu().numpy().astype(np.uint32)
    assert s[2] & 2, s
    assert s[0] > 65536, s
    o = out.cpu().numpy()
    assert np.all(o[cap:] == -7)
    written = o[: min(cap, int(s[1]))].astype(np.uint64)
    assert np.all(np.diff(written.astype(np.int64)) > 0)
    # every written code is a true motif of the single sequence (within d of one of its l-mers)
    import oracle
    orc = oracle.Oracle()
    for k in written[:50]:
        assert orc.is_motif(orc.decode(int(k), l), seqs, d)


def test_noalloc_few_ctas_matches_device_entry_point():
    # n = 64, m = 1100: the masks and planes leave room in the 16 MiB array for
    # the row scratch of only a few CTAs; the result must not depend on that
    import torch
    lib = pms.load()
    stream = torch.cuda.Stream()
    ctx = pms.Context(0)
    ctx.set_stream(stream)
    inst = pi.planted_instance(64, 1100, 15, 4, 93)
    cap = 4096
    for _ in range(2):
        with torch.cuda.stream(stream):
            want_st, want = _reference(ctx, torch, inst.seqs, inst.l, inst.d, cap)
            got_st, got = _noalloc(lib, torch, stream, inst.seqs, inst.l, inst.d, cap)
        assert got_st[2] == want_st[2] == 0
        assert np.array_equal(got, want)
        assert pi_key(inst.motif) in set(int(k) for k in got)
    ctx.close()


def pi_key(motif: bytes) -> int:
    k = 0
    for ch in motif.decode():
        k = 4 * k + "ACGT".index(ch)
    return k
