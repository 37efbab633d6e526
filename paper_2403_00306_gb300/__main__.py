"""Command line: solve one seeded synthetic planted-motif instance on the GPU.

    python -m paper_2403_00306_gb300 --l 15 --d 4 [--n 20 --m 600 --seed 1 --repeat 1 --count]
                                     [--opt grab=1 --opt partial_rows=-1 ...] [--alphabet protein]

Prints the motifs found and the solve's counters/timings (JSON). Used, for
instance, as the target of ncu captures of one solve.
"""
import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import planted_inputs as pi  # noqa: E402
import paper_2403_00306_gb300 as pms  # noqa: E402


def main() -> None:
    ap = argparse.ArgumentParser(prog="python -m paper_2403_00306_gb300")
    ap.add_argument("--l", type=int, required=True)
    ap.add_argument("--d", type=int, required=True)
    ap.add_argument("--n", type=int, default=20)
    ap.add_argument("--m", type=int, default=600)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--count", action="store_true", help="also count comparisons (count-mode kernel)")
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--alphabet", default=None,
                    help="general-alphabet search (pms_solve_sigma): 'protein' for the twenty amino acids, "
                         "or the letters themselves")
    ap.add_argument("--opt", action="append", default=[], metavar="NAME=VALUE",
                    help="set a pms_options field (repeatable)")
    a = ap.parse_args()
    opts = {}
    for kv in a.opt:
        k, v = kv.split("=", 1)
        opts[k] = int(v)
    alphabet = None
    if a.alphabet:
        alphabet = pi.PROTEIN if a.alphabet == "protein" else a.alphabet.encode()
        inst = pi.planted_instance_sigma(a.n, a.m, a.l, a.d, a.seed, alphabet)
    else:
        inst = pi.planted_instance(a.n, a.m, a.l, a.d, a.seed)
    with pms.Context(a.device) as ctx:
        if a.count:
            opts["count_work"] = 1
        if opts:
            ctx.set_options(**opts)
        for _ in range(a.repeat):
            if alphabet:
                rows = ctx.solve_sigma(inst.seqs, a.l, a.d, alphabet)
                motifs = [bytes(r).decode() for r in rows[:20]]
                count = len(rows)
            else:
                codes = ctx.solve(inst.seqs, a.l, a.d)
                motifs = pms.decode_all(codes[:20], a.l)
                count = len(codes)
        stats = ctx.stats()
    print(json.dumps({"l": a.l, "d": a.d, "n": a.n, "m": a.m, "seed": a.seed,
                      "planted": inst.motif.decode(), "motifs": motifs, "count": count, "stats": stats}))


if __name__ == "__main__":
    main()
