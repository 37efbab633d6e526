"""Failure paths, with the failures made on the host (pms_inject_fault, pms_cancel): no GPU
fault, trap or hang is involved. Each test checks that the error code reaches the caller and
that the context, and every other request, still gives the right answer.

Covered here: a device allocation that fails, an upload that fails in the middle of a served
stream and in a batch, a request cancelled while queued. The memory budget running out and a
wait shorter than the work are covered in test_gpu_served.py.
"""
import time

import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms

pytestmark = pytest.mark.gpu


def test_allocation_failure_surfaces_and_the_context_recovers():
    inst = pi.plain_instance(15, 4, seed=7)
    ref = pms.Context(0)
    want = ref.solve(inst.seqs, 15, 4)
    ref.close()
    c = pms.Context(0)
    # a fresh context allocates its buffers on the first solve: the first two
    # allocation attempts (the sized one and its exact-size retry) fail
    c.inject_fault(pms.PMS_FAULT_ALLOC, after=0, count=2)
    with pytest.raises(pms.PMSError) as e:
        c.solve(inst.seqs, 15, 4)
    assert e.value.code == pms.PMS_ENOMEM
    assert "allocation" in c.last_error()
    assert np.array_equal(c.solve(inst.seqs, 15, 4), want)
    c.close()


def test_upload_failure_in_a_batch_and_the_next_batch():
    insts = pi.batch_instances(count=6, master_seed=31)
    batch = [(i.seqs, i.l, i.d) for i in insts]
    ref = pms.Context(0)
    want = ref.solve_batch(batch)
    ref.close()
    c = pms.Context(0)
    c.inject_fault(pms.PMS_FAULT_UPLOAD, after=0, count=1)
    with pytest.raises(pms.PMSError) as e:
        c.solve_batch(batch)
    assert e.value.code == pms.PMS_ECUDA
    for w, r in zip(want, c.solve_batch(batch)):
        assert np.array_equal(r, w)
    c.close()


def _served_mix(count, seed):
    return [inst for _, inst in pi.serve_requests(count=count, master_seed=seed, m_range=(200, 400))]


def test_upload_failure_mid_stream_fails_only_that_request():
    reqs = _served_mix(8, 41)
    ref = pms.Context(0)
    want = [ref.solve(r.seqs, r.l, r.d) for r in reqs]
    ref.close()
    c = pms.Context(0)
    c.inject_fault(pms.PMS_FAULT_UPLOAD, after=3, count=1)   # the fourth admitted request
    tickets = [c.submit(r.seqs, r.l, r.d) for r in reqs]
    failed = []
    for k, (t, w) in enumerate(zip(tickets, want)):
        try:
            got = c.wait(t, 60000)
            assert np.array_equal(got, w), k
        except pms.PMSError as e:
            assert e.code == pms.PMS_ECUDA
            failed.append(k)
        c.release(t)
    assert failed == [3]
    c.close()


def test_cancel_a_queued_request():
    # one request on the device at a time, and a long one first (tens of milliseconds):
    # the later ones queue behind it
    long_one = pi.planted_instance(20, 1200, 19, 6, 3)
    reqs = _served_mix(4, 43)
    ref = pms.Context(0)
    want = [ref.solve(r.seqs, r.l, r.d) for r in reqs]
    ref.close()
    c = pms.Context(0)
    c.set_options(serve_max_inflight=1)
    t0 = c.submit(long_one.seqs, 19, 6)
    tickets = [c.submit(r.seqs, r.l, r.d) for r in reqs]
    c.cancel(tickets[2])                     # queued behind three others
    time.sleep(0.005)                        # the scheduler admits the long request at once
    with pytest.raises(pms.PMSError) as e:
        c.cancel(t0)                         # on the device: it runs to completion
    assert e.value.code == pms.PMS_EBUSY
    with pytest.raises(pms.PMSError) as e:
        c.cancel(987654321)
    assert e.value.code == pms.PMS_ENOTFOUND
    c.wait(t0, 60000)
    c.release(t0)
    for k, (t, w) in enumerate(zip(tickets, want)):
        if k == 2:
            with pytest.raises(pms.PMSError) as e:
                c.wait(t, 60000)
            assert e.value.code == pms.PMS_ECANCELED
        else:
            assert np.array_equal(c.wait(t, 60000), w), k
        c.cancel(t)                          # finished (or withdrawn): a no-op
        c.release(t)
    c.close()


def test_fault_injection_arguments():
    c = pms.Context(0)
    with pytest.raises(pms.PMSError):
        c.inject_fault(7)
    with pytest.raises(pms.PMSError):
        c.inject_fault(pms.PMS_FAULT_ALLOC, after=-1)
    c.inject_fault(pms.PMS_FAULT_ALLOC, count=0)     # clears
    c.close()
