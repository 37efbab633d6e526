"""Served form (continuous batching): each request's result equals the plain solve of the same
instance run alone, with requests overlapping on the device; timeouts, release and admission limits."""
import time

import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms
from parity_helpers import py_key

pytestmark = pytest.mark.gpu


def _requests(count, seed):
    # the served mix: (l, d) in {(13,4), (15,4), (17,5)}, n = 20, m in [200, 1200]; shorter m keeps the test quick
    out = []
    for t, inst in pi.serve_requests(count=count, master_seed=seed, m_range=(200, 500)):
        out.append(inst)
    return out


def test_served_results_equal_alone_results():
    reqs = _requests(24, 7)
    plain = pms.Context(0)
    alone = [plain.solve(r.seqs, r.l, r.d) for r in reqs]
    ctx = pms.Context(0)
    tickets = [ctx.submit(r.seqs, r.l, r.d) for r in reqs]      # all arrive while earlier ones run
    for r, t, want in zip(reqs, tickets, alone):
        got = ctx.wait(t, 60000)
        assert np.array_equal(got, want), (r.l, r.d, r.m)
        assert py_key(r.motif.decode()) in set(int(k) for k in got)
        ctx.release(t)
    s = ctx.stats()
    assert s["serve_waves"] >= 1
    assert s["serve_overlapped_waves"] >= 1 and s["serve_max_requests_per_wave"] >= 2
    ctx.close()
    plain.close()


def test_served_admission_limit_and_poisson_arrivals():
    reqs = _requests(16, 11)
    plain = pms.Context(0)
    alone = [plain.solve(r.seqs, r.l, r.d) for r in reqs]
    ctx = pms.Context(0)
    ctx.set_options(serve_max_inflight=3, serve_wave_items=4)   # few slots, short waves
    tickets = []
    for r in reqs:
        tickets.append(ctx.submit(r.seqs, r.l, r.d))
        time.sleep(0.002)
    for t, want in zip(tickets, alone):
        assert np.array_equal(ctx.wait(t, 60000), want)
    ctx.close()
    plain.close()


def test_served_timeout_and_release():
    ctx = pms.Context(0)
    inst = pi.planted_instance(20, 1200, 17, 5, 3)
    t = ctx.submit(inst.seqs, 17, 5)
    with pytest.raises(pms.PMSError) as e:
        ctx.wait(t, 0)
    assert e.value.code == pms.PMS_ETIMEDOUT
    with pytest.raises(pms.PMSError) as e:
        ctx.release(t)
    assert e.value.code == pms.PMS_EBUSY
    got = ctx.wait(t, 60000)
    assert py_key(inst.motif.decode()) in set(int(k) for k in got)
    ctx.release(t)
    with pytest.raises(pms.PMSError) as e:
        ctx.release(t)
    assert e.value.code == pms.PMS_ENOTFOUND
    with pytest.raises(pms.PMSError) as e:
        ctx.wait(12345, 0)
    assert e.value.code == pms.PMS_ENOTFOUND
    bad = inst.seqs.copy()
    bad[2, 2] = ord("X")
    with pytest.raises(pms.PMSError) as e:
        ctx.submit(bad, 17, 5)
    assert e.value.code == pms.PMS_EINVAL
    ctx.close()


def test_memory_budget_enforced():
    c = pms.Context(0, mem_budget_bytes=1 << 20)
    inst = pi.plain_instance(15, 4, seed=2)
    with pytest.raises(pms.PMSError) as e:
        c.solve(inst.seqs, 15, 4)
    assert e.value.code == pms.PMS_ENOMEM
    c.close()
