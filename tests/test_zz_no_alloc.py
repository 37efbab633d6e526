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
