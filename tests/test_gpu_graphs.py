"""Captured CUDA graphs of one-instance and batched solves: replays give the same motif
sets as kernel-by-kernel launches, with each call's own input and output buffers, also
after the context's buffers were reallocated by a larger instance. Replays carry the
device-time events only when pms_options.graph = 1."""
import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms

pytestmark = pytest.mark.gpu


def _device_solve(ctx, torch, seqs, l, d, cap=4096):
    n, m = seqs.shape
    d_in = torch.from_numpy(seqs.copy()).cuda()
    out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    ctx.set_stream(torch.cuda.current_stream())     # ordered after the tensors' fills
    ctx.solve_device(d_in, n, m, l, d, out, cap, st)
    torch.cuda.synchronize()
    s = st.cpu().numpy().astype(np.uint32)
    assert s[2] == 0
    return out[: int(s[1])].cpu().numpy().astype(np.uint64)


def test_graph_replays_match_kernel_by_kernel(oracle_):
    torch = pytest.importorskip("torch")
    g = pms.Context(0)
    k = pms.Context(0)
    k.set_options(graph=-1)
    g.set_stream(torch.cuda.current_stream())
    k.set_stream(torch.cuda.current_stream())
    for (l, d) in [(15, 4), (9, 2)]:
        for seed in (1, 2, 3, 4):
            inst = pi.plain_instance(l, d, seed=seed)
            want = k.solve(inst.seqs, l, d)
            assert np.array_equal(g.solve(inst.seqs, l, d), want)
            # new input and output tensors on every call
            before = g.stats()["graph_replays"]
            assert np.array_equal(_device_solve(g, torch, inst.seqs, l, d), want)
            if g.stats()["graph_replays"] > before:
                # a replay without timing events reports no device times
                assert g.stats()["ms_verify"] == -1.0
            else:
                assert g.stats()["ms_verify"] > 0
    small = pi.planted_instance(6, 80, 9, 2, 5)
    assert np.array_equal(g.solve(small.seqs, 9, 2), oracle_.solve(small.seqs, 9, 2))
    g.close()
    k.close()


def test_graph_after_buffer_reallocation():
    torch = pytest.importorskip("torch")
    g = pms.Context(0)
    k = pms.Context(0)
    k.set_options(graph=-1)
    a = pi.planted_instance(8, 100, 11, 3, 7)
    b = pi.planted_instance(30, 1000, 13, 4, 8)     # larger: the context's buffers grow
    want_a, want_b = k.solve(a.seqs, 11, 3), k.solve(b.seqs, 13, 4)
    for _ in range(2):
        assert np.array_equal(g.solve(a.seqs, 11, 3), want_a)
    assert np.array_equal(g.solve(b.seqs, 13, 4), want_b)
    for _ in range(2):
        assert np.array_equal(g.solve(a.seqs, 11, 3), want_a)
        assert np.array_equal(_device_solve(g, torch, a.seqs, 11, 3), want_a)
    g.close()
    k.close()


def test_batch_graph_replays_match_kernel_by_kernel():
    # a batch of uneven instances: the first call runs kernel by kernel, the second is
    # captured, later calls replay the graph (the replay counter says so)
    insts = pi.batch_instances(count=12, master_seed=99)
    batch = [(i.seqs, i.l, i.d) for i in insts]
    k = pms.Context(0)
    k.set_options(graph=-1)
    want = k.solve_batch(batch)
    g = pms.Context(0)
    before = g.stats()["graph_replays"]
    for call in range(4):
        got = g.solve_batch(batch)
        for w, r in zip(want, got):
            assert not isinstance(r, Exception) and np.array_equal(r, w), call
    assert g.stats()["graph_replays"] - before == 2
    # another batch shape does not replay the first one's graph
    other = batch[:5]
    got = g.solve_batch(other)
    for w, r in zip(k.solve_batch(other), got):
        assert np.array_equal(r, w)
    assert g.stats()["graph_replays"] - before == 2
    g.close()
    k.close()


def test_timed_graph_replays():
    # graph = 1: the device-time events are nodes of the graph, so replays report the
    # verification kernel's time; the motif sets are those of the untimed replays
    torch = pytest.importorskip("torch")
    t = pms.Context(0)
    t.set_options(graph=1)
    u = pms.Context(0)
    for seed in (1, 2, 3):
        inst = pi.plain_instance(15, 4, seed=seed)
        for call in range(3):
            got = _device_solve(t, torch, inst.seqs, 15, 4)
            s = t.stats()
            assert s["ms_verify"] > 0 and s["ms_kernel"] >= s["ms_verify"], (seed, call)
            assert np.array_equal(got, _device_solve(u, torch, inst.seqs, 15, 4))
    assert t.stats()["graph_replays"] >= 4 and u.stats()["graph_replays"] >= 4
    # a solve launched kernel by kernel (count mode never replays) is always timed
    u.set_options(count_work=1)
    u.solve(pi.plain_instance(15, 4, seed=1).seqs, 15, 4)
    assert u.stats()["ms_verify"] > 0
    t.close()
    u.close()


def test_graph_option_values():
    c = pms.Context(0)
    c.set_options(graph=-1)
    c.set_options(graph=0)
    c.set_options(graph=1)
    with pytest.raises(pms.PMSError):
        c.set_options(graph=-2)
    c.close()
