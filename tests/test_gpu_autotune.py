"""Autotuner: tuned schedules change only speed, never the motif set; the table round-trips."""
import numpy as np
import pytest

import planted_inputs as pi
import paper_2403_00306_gb300 as pms

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results(tmp_path):
    base = pms.Context(0)
    ctx = pms.Context(0)
    t = ctx.autotune(20, 600, 13, 4)
    assert t["ms"] > 0 and 1 <= t["prune_rows"] <= 19 and t["chunk_work"] > 0 and t["ctas_per_sm"] >= 1
    for seed in (1, 2):
        inst = pi.plain_instance(13, 4, seed=seed)
        assert np.array_equal(ctx.solve(inst.seqs, 13, 4), base.solve(inst.seqs, 13, 4))
    path = tmp_path / "tuning.txt"
    ctx.save_tuning(str(path))
    text = path.read_text().splitlines()
    assert any(line.startswith("13 4 32 1024 ") for line in text)
    other = pms.Context(0)
    other.load_tuning(str(path))
    inst = pi.plain_instance(13, 4, seed=3)
    assert np.array_equal(other.solve(inst.seqs, 13, 4), base.solve(inst.seqs, 13, 4))
    for c in (base, ctx, other):
        c.close()


def test_autotune_option_on_batch():
    insts = pi.batch_instances(count=12, master_seed=99)
    base = pms.Context(0)
    want = [base.solve(i.seqs, i.l, i.d) for i in insts]
    ctx = pms.Context(0)
    ctx.set_options(autotune=1)
    got = ctx.solve_batch([(i.seqs, i.l, i.d) for i in insts])
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    base.close()
    ctx.close()
