"""Autotuner of the launch plans (kernel, tile variant, j-splits) of the regular-force step.

For a particle count n and each active-block size bucket (powers of two up to n), every
candidate plan is run through the plan override of the C ABI (nb_set_plan_override) and
timed with the library's own device timers (nb_get_timings, CUDA events on the launch
stream); the fastest becomes the bucket's entry of a plan table (nb_set_plan_table), except
that a staged-hit variant within 1 % of it (a tie at the run-to-run spread) is preferred for
its lower DRAM traffic.  The
table is stored as JSON keyed by GPU name, SM count, precision and n bucket, so a run on
the same kind of device installs it without re-tuning (Context.apply_tuned()).

The batched ensemble form is tuned the same way over its tile variants (tune_batched).

Usage (on a GPU): python -m paper_1504_03687_gb300.tune --n 1048576 [--prec mixed] [--max-ni 32]
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np

TABLE_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_plans.json")

# candidate plans: (kernel, variant, splits); splits 0 = the planner's split count
MIXED_CANDIDATES = [(1, v, 0) for v in range(20)] + [(2, v, 0) for v in range(4)]
# the mixed variants that stage their neighbour hits and write them as whole groups (less
# DRAM traffic for the same lists); a plan within TIE of the fastest counts as a tie (the
# run-to-run spread of a call is about 1 %), and a tie goes to the fastest of these
STAGED_VARIANTS = (15, 16, 17, 18, 19)
TIE = 0.01
FP64_CANDIDATES = [(0, 0, 0), (3, 0, 0), (3, 1, 0)]


def device_key(precision: str, n: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sms={p.multi_processor_count}|{precision}|n=2^{int(round(math.log2(max(n, 1))))}"


def choose_plan(timed):
    """The table entry from [(plan, ms), ...]: the fastest plan, or the fastest staged-hit
    variant if it is within TIE of it."""
    best = min(timed, key=lambda e: e[1])
    staged = [e for e in timed if e[0][0] == 1 and e[0][1] in STAGED_VARIANTS and e[1] <= best[1] * (1 + TIE)]
    return min(staged, key=lambda e: e[1]) if staged else best


def _time_plan(ctx, idx, rs2, plan, reps):
    ctx.set_plan_override(*plan)
    ctx.regular_force(idx, rs2, neighbours=True)  # warm-up (and scratch growth)
    ctx.sync()
    ctx.timings()
    ctx.set_timing(True)
    for _ in range(reps):
        ctx.regular_force(idx, rs2, neighbours=True)
    ph = ctx.timings()
    ctx.set_timing(False)
    ctx.sync()
    ctx.set_plan_override(-1)
    # the anchored variants pay for their row order too
    return (ph["order"][0] + ph["force"][0] + ph["reduce"][0] + ph["neighbours"][0]) / reps


def tune_force(ctx, order, rs2, buckets=None, reps=2, candidates=None, log=print):
    """Time every candidate plan for blocks of the sizes in `buckets` (the head of the
    sorted step list `order`); returns [(ni_max, kernel, variant, splits, ms), ...]."""
    import torch
    n = ctx.n
    if buckets is None:
        buckets = [1 << k for k in range(0, int(math.log2(n)) + 1)]
    if candidates is None:
        candidates = MIXED_CANDIDATES if ctx.precision == "mixed" else FP64_CANDIDATES
    dev = torch.device("cuda", ctx.device)
    rs2_t = torch.tensor([rs2], dtype=torch.float64, device=dev)
    table = []
    for ni in buckets:
        idx = torch.as_tensor(np.ascontiguousarray(order[:ni].astype(np.int32)), device=dev)
        timed = []
        for plan in candidates:
            if plan[0] in (2, 3) and ni > 256:
                continue  # the j-streamed kernels are for small blocks only
            try:
                ms = _time_plan(ctx, idx, rs2_t, plan, reps)
            except Exception as exc:  # a plan the context rejects is skipped
                log(f"  n_i={ni} plan={plan}: skipped ({exc})")
                continue
            timed.append((plan, ms))
        best = choose_plan(timed)
        log(f"n_i={ni}: best {best[0]} {best[1]:.4f} ms ({ni * n / best[1] / 1e6:.1f} Ginteractions/s)")
        table.append((ni, best[0][0], best[0][1], best[0][2], best[1]))
    return table


def tune_batched(ctx, cluster_off, active_off, idx, rs2, reps=3, log=print):
    """Best tile variant of the batched form for this ensemble -> (variant, ms per launch)."""
    import torch
    best = None
    for v in range(3):
        ctx.batch_plan(cluster_off, active_off, v)
        out = ctx.regular_force_batched(idx, rs2)
        ctx.sync()
        ctx.timings()
        ctx.set_timing(True)
        for _ in range(reps):
            ctx.regular_force_batched(idx, rs2, out=out)
        ph = ctx.timings()
        ctx.set_timing(False)
        ms = (ph["force"][0] + ph["reduce"][0] + ph["neighbours"][0]) / reps
        log(f"batched variant {v}: {ms:.3f} ms")
        if best is None or ms < best[1]:
            best = (v, ms)
    torch.cuda.synchronize()
    return best


def load_table(key: str, path: str = TABLE_FILE):
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f).get(key)


def save_table(key: str, table, path: str = TABLE_FILE):
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[key] = [list(map(float, e[:1])) + list(e[1:4]) + [float(e[4])] for e in table]
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def merge_table(old, new):
    """The stored table with the buckets of `new` replaced (or added), in bucket order: a
    re-tune of some buckets keeps the entries of the others."""
    keep = {float(e[0]): list(e) for e in (old or [])}
    for e in new:
        keep[float(e[0])] = [float(e[0])] + list(e[1:4]) + [float(e[4])]
    return [keep[k] for k in sorted(keep)]


def apply_table(ctx, table):
    """Install a tuned table: bucket b covers (previous bucket, b]; the last bucket covers
    every larger block as well."""
    entries = []
    for q, e in enumerate(table):
        ni_max = int(e[0]) if q + 1 < len(table) else 1 << 62
        entries.append((ni_max, int(e[1]), int(e[2]), int(e[3])))
    ctx.set_plan_table(entries)


def main():
    import torch

    import workloads as W
    from paper_1504_03687_gb300 import Context
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=TABLE_FILE)
    ap.add_argument("--max-ni", type=int, default=0,
                    help="re-tune only the buckets up to this block size and keep the stored others")
    args = ap.parse_args()
    cl = W.king(args.n, 2, W0=6.0, masses="kroupa", binary_fraction=0.05)
    rs2 = W.neighbour_radius2(cl.x, 80, seed=2)
    order = W.sorted_step_list(W.block_steps(cl, seed=2))
    dev = torch.device("cuda", 0)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    ctx = Context(cl.n, precision=args.prec, nb_cap=512)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    buckets = [1 << k for k in range(0, int(math.log2(cl.n)) + 1, 1)]
    if args.prec == "fp64":
        buckets = [b for b in buckets if b <= 1 << 14]
    if args.max_ni > 0:
        buckets = [b for b in buckets if b <= args.max_ni]
    table = tune_force(ctx, order, rs2, buckets=buckets, reps=args.reps)
    key = device_key(args.prec, cl.n)
    if args.max_ni > 0:
        table = merge_table(load_table(key, args.out), table)
    save_table(key, table, args.out)
    print(json.dumps({"key": key, "table": table}))


if __name__ == "__main__":
    main()
