#!/usr/bin/env python
"""Benchmark of the regular-force step on one or more GB300s.

One step = one regular-force block cycle on the million-body workload: for each
active block of 2^10, 2^14, 2^17 and 2^20 particles (the sorted time-step list of a
King W0 = 6 cluster of 2^20 j-particles incl. 5% binary centre-of-mass particles,
Kroupa masses), predict all particles to the block time (FP64) and compute the mixed-
precision force, jerk, potential and CSR neighbour lists (r_s for a median of 80,
cap 512).  value = pairs (N_i x N summed over the blocks) / device time, in
Ginteractions/s; 60 flops per pair gives the FP32 roofline fraction.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own seeded cluster (independent problems, weak
scaling, no collective in the step); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "force+jerk Ginteractions/s & %FP32 peak at N=2^20, mixed vs FP64, at stated error"
UNIT = "Ginteractions/s"
FLOPS_PER_PAIR = 60
BLOCKS = (1 << 10, 1 << 14, 1 << 17, 1 << 20)
NB_CAP = 512

# DRAM bytes (read + write) of the four force launches of one step (blocks 2^10 .. 2^20), from
# one ncu capture of `bench.py --steps 1 --warmup 3 --no-e2e --no-cpu --no-ensemble
# --no-adjoint --no-irregular --no-scheduler --no-integrator` (metrics dram__bytes_read.sum,
# dram__bytes_write.sum; -s 12 -c 4: the timed step's launches), valid only for the
# force-kernel sources whose SHA-256 is recorded with them (FORCE_SOURCES: the kernels, their
# device helpers and their argument header).
FORCE_TRAFFIC = {"sources_sha256": "3af94ab8688af704dc2a434cae013cb3e265cf9e64425017717da68e9a09c748",
                 "bytes_per_launch": [55140864, 119358976, 431456768, 1169148672]}
FORCE_SOURCES = ("force_mixed.cu", "nb_common.cuh", "nb_force.cuh", "roworder.cu")


def force_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1504_03687_gb300", "csrc")
    for f in FORCE_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def force_traffic_per_launch():
    """Mean DRAM bytes per force launch of a step, or None if the kernel sources changed
    since the counters were taken."""
    rec = FORCE_TRAFFIC
    if rec["bytes_per_launch"] is None or rec["sources_sha256"] != force_sources_sha256():
        return None
    return sum(rec["bytes_per_launch"]) / len(rec["bytes_per_launch"])
NB_PER_ROW = NB_CAP  # CSR capacity per active particle: room for every list at the cap
WORKLOAD = ("King W0=6, N=2^20 j-particles (5% binary c.m.), Kroupa IMF, N-body units; "
            "active blocks 2^10/2^14/2^17/2^20 from the sorted step list; "
            "predict + mixed regular force + neighbour CSR per block")


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def build_workload(seed):
    import workloads as W
    cl, rs2 = W.king_1m_binaries(seed=seed)
    steps = W.block_steps(cl, seed=seed)
    order = W.sorted_step_list(steps).astype(np.int32)
    a0, j0, tl = W.hermite_state(cl, seed=seed, t_block=0.125, steps=steps)
    return cl, rs2, order, a0, j0, tl


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "sm_mhz_min": min(sm) if sm else None,
                "power_w_max": max(pw) if pw else None}


def fp32_peak_tflops(num_sms):
    """FP32 CUDA-core peak: SMs x 128 lanes x 2 flops (FMA) x maximum SM clock."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
        src = "SMs x 128 FP32 lanes x 2 x sm_max_mhz of MEASURED_PEAKS.json"
    except (OSError, ValueError):
        src = "SMs x 128 FP32 lanes x 2 x 2070 MHz (nominal maximum SM clock)"
    return num_sms * 128 * 2 * mhz * 1e6 / 1e12, src


def host_cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine architecture."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip() + " (" + platform.machine() + ")"
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def oracle_rate(cl, rs2, rows, threads=None):
    """Oracle pairs/s on `rows` active particles against all j (host cores)."""
    import oracle
    if threads:
        oracle.set_num_threads(threads)
    t0 = time.perf_counter()
    oracle.regular_force(cl.x, cl.v, cl.m, rows, rs2, cap=NB_CAP, lists=False)
    dt = time.perf_counter() - t0
    return rows.size * cl.n / dt, dt


def run_reference(args):
    """The oracle as it stands, on the host cores, on a bounded sample of the workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    cl, rs2, order, a0, j0, tl = build_workload(seed=2)
    xp, vp = oracle.predict(0.125, cl.x, cl.v, a0, j0, tl)
    cl.x, cl.v = xp, vp
    rate, _ = oracle_rate(cl, rs2, order[:16])
    rows = int(max(16, min(1 << 20, 6.0 * rate / cl.n)))  # ~6 s of oracle work per step
    sample = order[:rows]
    for _ in range(args.warmup):
        oracle_rate(cl, rs2, sample)
    tot, pairs = 0.0, 0
    for _ in range(args.steps):
        r, dt = oracle_rate(cl, rs2, sample)
        tot += dt
        pairs += rows * cl.n
    value = pairs / tot / 1e9
    cores = oracle.num_threads()
    sample_desc = (f"{rows} active rows (head of the sorted step list) x all {cl.n} j per step, "
                   "FP64 direct sum with neighbour lists")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": cl.n, "sample": sample_desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc,
                         "cpu": host_cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-irregular", action="store_true")
    ap.add_argument("--no-scheduler", action="store_true")
    ap.add_argument("--no-integrator", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="profiling case: one warm-up and one timed predict + force call on the King cluster "
                         "(--n particles, --ni active, --prec), printing device times")
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--ni", type=int, default=2048)
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--backward", action="store_true", help="with --profile: also run the adjoint")
    ap.add_argument("--no-lists", action="store_true",
                    help="with --profile: the force call without neighbour capture (sums only)")
    ap.add_argument("--irregular", action="store_true",
                    help="with --profile: also run the irregular force over the lists just returned")
    ap.add_argument("--model", default="king", choices=["king", "plummer"],
                    help="with --profile: King W0=6 (+5%% binaries) or Plummer, Kroupa masses")
    ap.add_argument("--variants", default="",
                    help="with --profile: comma list of kernel:variant:splits plans to time in turn "
                         "(e.g. 1:0:14,1:5:14); empty = the automatic plan")
    ap.add_argument("--ac-plummer", action="store_true",
                    help="only the mixed Ahmad-Cohen integration of the 65536-body Plummer sphere to t = 1/64 "
                         "(the ac_integrator.mixed run); prints its JSON line")
    ap.add_argument("--ac-king", type=float, default=None, metavar="T_END",
                    help="only the Ahmad-Cohen integration of the million-body King cluster, from t = 0 to "
                         "T_END (steps at most min(T_END, 1/64)); prints its JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile_case(args)
    if args.ac_plummer:
        import torch
        print(json.dumps(bench_ac(torch.device("cuda", 0), precisions=("mixed",), reference=False)))
        return
    if args.ac_king is not None:
        import torch
        dev = torch.device("cuda", 0)
        print(json.dumps(bench_ac_king_1m(dev, t_end=args.ac_king, dt_max=min(args.ac_king, 1.0 / 64))))
        return

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1504_03687_gb300 import Context

    # one problem for every rank: the copy algorithm shares each block's rows among the ranks
    cl, rs2, order, a0, j0, tl = build_workload(seed=2)
    n = cl.n
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    state = [T(q) for q in (cl.x, cl.v, a0, j0, cl.m, tl)]
    idx_dev = [T(order[:b]) for b in BLOCKS]
    rs2_dev = torch.tensor([rs2], dtype=torch.float64, device=dev)
    ctx = Context(n, precision="mixed", nb_cap=NB_CAP, device=local)
    ctx.set_particles(*state)
    tuned = ctx.apply_tuned()  # launch plans from the autotuner's table for this GPU, if any
    outs = [None] * len(BLOCKS)

    share = [None] * len(BLOCKS)  # this rank's row results of every block (copy algorithm)

    def force_rows(q):
        def run(rows):
            ctx.predict(0.125)
            share[q] = ctx.regular_force(rows, rs2_dev, nb_capacity=rows.shape[0] * NB_PER_ROW, out=share[q])
            r = share[q]
            return r.acc, r.jerk, r.pot, r.nb_off, r.nb_idx
        return run

    def step():
        if world == 1:
            for q, b in enumerate(BLOCKS):
                ctx.predict(0.125)
                outs[q] = ctx.regular_force(idx_dev[q], rs2_dev, nb_capacity=b * NB_PER_ROW, out=outs[q])
        else:
            res = copy_algorithm_step(idx_dev, [force_rows(q) for q in range(len(BLOCKS))], world, rank)
            for q, r in enumerate(res):
                outs[q] = GatheredBlock(*r)

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    pairs_step = sum(BLOCKS) * n
    for _ in range(args.warmup):
        step()
    ctx.sync()
    ctx.timings()  # reset counters
    ctx.set_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xff)  # L2 flush between timed steps (outside the events)
        ev[k][0].record()
        step()
        ev[k][1].record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ctx.set_timing(False)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    phase = ctx.timings()
    ctx.sync()
    ms_t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    # one problem's pairs: with several ranks each computed a share of every block's rows
    value = pairs_step * args.steps / (ms_max * 1e-3) / 1e9
    launches = int(sum(v[1] for v in phase.values()))
    force_ms = phase["force"][0]
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_src = fp32_peak_tflops(num_sms)
    # the force kernel of this rank computed its share of every block's rows
    from paper_1504_03687_gb300.dist import shard_rows
    pairs_rank = sum((lambda lh: lh[1] - lh[0])(shard_rows(b, world, rank)) for b in BLOCKS) * n
    achieved = FLOPS_PER_PAIR * pairs_rank * args.steps / (force_ms * 1e-3) / 1e12

    # end to end through the public API with host buffers (pinned), copies inside the timing;
    # measured right after the device-timed steps, before the other sections load the GPU
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory().numpy()
        h_state = [pin(q) for q in (cl.x, cl.v, a0, j0, cl.m, tl)]
        h_idx = [pin(order[:b]) for b in BLOCKS]
        h_out = []
        for b in BLOCKS:
            from paper_1504_03687_gb300.api import ForceResult
            h_out.append(ForceResult(acc=pin(np.empty((b, 3))), jerk=pin(np.empty((b, 3))), pot=pin(np.empty(b)),
                                     nb_off=pin(np.empty(b + 1, np.int64)),
                                     nb_idx=pin(np.empty(b * NB_PER_ROW, np.int32)),
                                     nb_count=pin(np.empty(b, np.int32))))
        h2d = sum(q.nbytes for q in h_state) + sum(q.nbytes for q in h_idx) + 8 * len(BLOCKS)

        # one GPU: the step's inputs go up, the blocks run on the device largest first, and each
        # block's results come down on a copy stream while the next block computes (the copies
        # of the largest block's 1 GB of lists hide behind the three smaller blocks)
        order_q = sorted(range(len(BLOCKS)), key=lambda q: -BLOCKS[q])
        d_idx_e = [torch.empty(b, dtype=torch.int32, device=dev) for b in BLOCKS]
        outs_e = [None] * len(BLOCKS)
        copy_stream = torch.cuda.Stream(device=dev)
        done_ev = [torch.cuda.Event() for _ in BLOCKS]

        def e2e_step():
            d2h = 0
            ctx.set_particles(*h_state)
            if world == 1:
                for q in order_q:
                    d_idx_e[q].copy_(torch.from_numpy(h_idx[q]), non_blocking=True)
                    ctx.predict(0.125)
                    outs_e[q] = ctx.regular_force(d_idx_e[q], rs2_dev, nb_capacity=BLOCKS[q] * NB_PER_ROW,
                                                  out=outs_e[q])
                    done_ev[q].record()
                with torch.cuda.stream(copy_stream):
                    for q in order_q:
                        copy_stream.wait_event(done_ev[q])
                        r, h = outs_e[q], h_out[q]
                        used = int(r.nb_off[-1:].to("cpu").item())  # waits for this block only
                        used = min(used, h.nb_idx.shape[0])
                        for hd, dv in ((h.acc, r.acc), (h.jerk, r.jerk), (h.pot, r.pot), (h.nb_off, r.nb_off),
                                       (h.nb_count, r.nb_count)):
                            torch.from_numpy(hd).copy_(dv, non_blocking=True)
                            d2h += hd.nbytes
                        torch.from_numpy(h.nb_idx[:used]).copy_(r.nb_idx[:used], non_blocking=True)
                        d2h += used * 4
                copy_stream.synchronize()
                ctx.sync()
                return d2h
            # several ranks: each computes its share of the rows from the host arrays, the shares
            # are exchanged on the device (NCCL) and every rank reads the whole block back
            def host_rows(q):
                def run(rows):
                    ctx.predict(0.125)
                    lo, hi = rows
                    host_force(ctx, h_idx[q][lo:hi], rs2, h_out[q])
                    return tuple(torch.as_tensor(np.ascontiguousarray(a[:k]), device=dev)
                                 for a, k in ((h_out[q].acc, hi - lo), (h_out[q].jerk, hi - lo),
                                              (h_out[q].pot, hi - lo), (h_out[q].nb_off, hi - lo + 1),
                                              (h_out[q].nb_idx, int(h_out[q].nb_off[hi - lo]))))
                return run
            from paper_1504_03687_gb300.dist import shard_rows
            spans = [shard_rows(b, world, rank) for b in BLOCKS]
            res = copy_algorithm_step([np.arange(b) for b in BLOCKS], [host_rows(q) for q in range(len(BLOCKS))],
                                      world, rank, shares=spans)
            for r in res:
                for t in r:
                    d2h += t.cpu().numpy().nbytes
            return d2h

        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e2e_clocks = ClockSampler(local)
        e2e_clocks.start()
        t0 = time.perf_counter()
        d2h = 0
        step_s = []
        for _ in range(args.steps):
            ts = time.perf_counter()
            d2h = e2e_step()
            step_s.append(time.perf_counter() - ts)  # host-mode calls return after their copies
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e_clk = e2e_clocks.stop()
        el_t = torch.tensor([el], dtype=torch.float64, device=dev)
        if world > 1:
            torch.distributed.all_reduce(el_t, op=torch.distributed.ReduceOp.MAX)
        e2e = {"value": pairs_step * args.steps / float(el_t.item()) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "step_ms": [round(x * 1e3, 2) for x in step_s], "clocks": e2e_clk}

    # accuracy at the stated error: sampled rows of the full block vs the FP64 oracle,
    # and the GPU FP64 path on the 2^14 block (the >= 3x comparison)
    # with more than one rank only the step itself (and its accuracy) is measured: the other
    # sections are single-GPU measurements and would hold every rank's GPU meanwhile
    solo = world == 1
    extra = {}
    if rank == 0:
        import oracle
        rng = np.random.default_rng(0)
        sel = np.sort(rng.choice(BLOCKS[-1], 64, replace=False))
        full = outs[-1]
        xp_np, vp_np = oracle.predict(0.125, cl.x, cl.v, a0, j0, tl)  # the oracle's own predictor
        rows = order[:BLOCKS[-1]][sel]
        ref = oracle.regular_force(xp_np, vp_np, cl.m, rows, rs2, cap=NB_CAP, lists=False)

        def errs(acc, jerk, pot):
            ea = np.linalg.norm(acc - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1)
            ej = np.linalg.norm(jerk - ref[1], axis=1) / np.linalg.norm(ref[1], axis=1)
            ep = np.abs(pot - ref[2]) / np.abs(ref[2])
            return {q: {"median": float(np.median(e)), "max": float(e.max())}
                    for q, e in (("acc", ea), ("jerk", ej), ("pot", ep))}
        extra["error_vs_oracle_mixed"] = errs(full.acc[sel].cpu().numpy(), full.jerk[sel].cpu().numpy(),
                                              full.pot[sel].cpu().numpy())
    if rank == 0 and solo:
        ctx64 = Context(n, precision="fp64", nb_cap=NB_CAP, device=local)
        ctx64.set_particles(*state)
        ctx64.predict(0.125)
        b64 = BLOCKS[1]
        out64 = ctx64.regular_force(idx_dev[1], rs2_dev, nb_capacity=b64 * NB_PER_ROW)
        ctx64.sync()
        ctx64.timings()
        ctx64.set_timing(True)
        reps = 2
        for _ in range(reps):
            out64 = ctx64.regular_force(idx_dev[1], rs2_dev, nb_capacity=b64 * NB_PER_ROW, out=out64)
        ph64 = ctx64.timings()
        ctx64.sync()
        fp64_rate = reps * b64 * n / (ph64["force"][0] * 1e-3) / 1e9
        ctx.set_timing(True)
        for _ in range(reps):
            ctx.regular_force(idx_dev[1], rs2_dev, nb_capacity=b64 * NB_PER_ROW, out=outs[1])
        ph32 = ctx.timings()
        ctx.set_timing(False)
        mixed_rate = reps * b64 * n / (ph32["force"][0] * 1e-3) / 1e9
        sel64 = np.sort(rng.choice(b64, 32, replace=False))
        ref = oracle.regular_force(xp_np, vp_np, cl.m, order[:b64][sel64], rs2, cap=NB_CAP, lists=False)
        extra["error_vs_oracle_fp64"] = errs(out64.acc[sel64].cpu().numpy(), out64.jerk[sel64].cpu().numpy(),
                                             out64.pot[sel64].cpu().numpy())
        extra["fp64_path"] = {"block": b64, "force_kernel_Ginteractions_s": fp64_rate,
                              "mixed_force_kernel_Ginteractions_s_same_block": mixed_rate,
                              "mixed_over_fp64": mixed_rate / fp64_rate}
        extra["small_blocks"] = bench_small_blocks(ctx, n, order, rs2_dev, dev)
        if not args.no_irregular:
            extra["irregular"] = bench_irregular(ctx, ctx64, cl, (a0, j0, tl), order, idx_dev, outs, rs2)
        if not args.no_scheduler:
            extra["scheduler"] = bench_scheduler(dev, cl)
        ctx64.close()

    if rank == 0 and solo and not args.no_ensemble:
        extra["ensemble"] = bench_ensemble(dev)
    if rank == 0 and solo and not args.no_adjoint:
        extra["adjoint"] = bench_adjoint(dev)
    if rank == 0 and solo and not args.no_integrator:
        extra["ac_integrator"] = bench_ac(dev)
    cpu = None
    if rank == 0 and solo and not args.no_cpu:
        import oracle
        import types
        xp_np, vp_np = oracle.predict(0.125, cl.x, cl.v, a0, j0, tl)
        pred = types.SimpleNamespace(x=xp_np, v=vp_np, m=cl.m, n=cl.n)
        rate, _ = oracle_rate(pred, rs2, order[:32])
        rows = int(max(32, min(BLOCKS[-1], 12.0 * rate / n)))  # ~12 s of oracle work
        rate, dt = oracle_rate(pred, rs2, order[:rows])
        cores = oracle.num_threads()
        cpu = {"value": rate / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": host_cpu_model(),
               "sample": f"{rows} active rows (head of the sorted step list) x all {n} j, FP64 direct sum "
                         f"with neighbour lists, {dt:.1f} s"}
        rate1, dt1 = oracle_rate(pred, rs2, order[:16], threads=1)  # the same oracle on one core
        oracle.set_num_threads(cores)
        cpu["single_core"] = {"value": rate1 / 1e9, "sample": f"16 active rows x all {n} j, {dt1:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (one seeded King W0=6 cluster, the same on every rank)",
            "config": {"workload": WORKLOAD, "n": n, "blocks": list(BLOCKS), "pairs_per_step": pairs_step,
                       "nb_cap": NB_CAP, "rs2": rs2, "precision": "mixed (ds-f32 differences, f32 pairwise, "
                       "f64 predictor and per-tile sums)", "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": ("one GPU" if world == 1 else
                                       f"row-sharded copy algorithm over {world} GPUs: every rank holds all "
                                       f"N, computes a contiguous share of each block's rows, NCCL all-gather "
                                       f"of the row results (acc, jerk, pot, CSR lists) inside the timing"),
                       "launch_plans": "autotuned table" if tuned else "automatic planner",
                       "accuracy": accuracy_summary(extra)},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": force_traffic_per_launch(),
                         "traffic_per_block": (dict(zip(map(str, BLOCKS), FORCE_TRAFFIC["bytes_per_launch"]))
                                               if force_traffic_per_launch() is not None else None),
                         "kernel": "force (mixed tiled / j-streamed)", "peak_source": peak_src,
                         "flops_per_pair": FLOPS_PER_PAIR, "force_kernel_ms_per_step": force_ms / args.steps},
            "fp32_peak_frac_whole_step": value * 1e9 * FLOPS_PER_PAIR / (peak * 1e12) / world,
            "phase_ms_per_step": {k: v[0] / args.steps for k, v in phase.items()},
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


class GatheredBlock:
    """A block's gathered row results (the fields of a force result that the bench reads)."""

    def __init__(self, acc, jerk, pot, nb_off, nb_idx):
        self.acc, self.jerk, self.pot, self.nb_off, self.nb_idx = acc, jerk, pot, nb_off, nb_idx


def copy_algorithm_step(blocks, forces, world, rank, shares=None, group=None):
    """One step of the copy algorithm (paper Sec. 3.1, the O(N_i) result exchange of Table 2):
    every rank holds all particles, computes the rows shard_rows(n_i, world, rank) of each
    active block with forces[q](rows) -> (acc, jerk, pot, nb_off, nb_idx), and the row results
    are all-gathered in rank order (dist.allgather_rows) so that every rank holds every block.
    blocks[q] are the blocks' active index lists; with `shares`, forces[q] is given the row
    span (lo, hi) instead of the rows themselves.  Returns the gathered blocks."""
    from paper_1504_03687_gb300.dist import allgather_rows, shard_rows
    out = []
    for q, rows in enumerate(blocks):
        lo, hi = shares[q] if shares is not None else shard_rows(int(rows.shape[0]), world, rank)
        res = forces[q]((lo, hi) if shares is not None else rows[lo:hi])
        out.append(allgather_rows(*res, group=group) if world > 1 else res)
    return out


def accuracy_summary(extra):
    """The stated-error and FP64-comparison figures in compact form ([median, max] relative error
    per particle against the FP64 oracle; mixed over FP64 force-kernel rate on the same block),
    kept inside the contract line's config."""
    out = {}
    for key, name in (("error_vs_oracle_mixed", "mixed_vs_oracle_64_rows_of_2^20_block"),
                      ("error_vs_oracle_fp64", "fp64_vs_oracle_32_rows_of_2^14_block")):
        if key in extra:
            out[name] = {q: [float(f"{v['median']:.3g}"), float(f"{v['max']:.3g}")] for q, v in extra[key].items()}
    if "fp64_path" in extra:
        f = extra["fp64_path"]
        out["fp64_Ginteractions_s_2^14_block"] = round(f["force_kernel_Ginteractions_s"], 2)
        out["mixed_Ginteractions_s_2^14_block"] = round(f["mixed_force_kernel_Ginteractions_s_same_block"], 1)
        out["mixed_over_fp64"] = round(f["mixed_over_fp64"], 1)
    return out


def run_profile_case(args):
    """Small, self-contained case for ncu captures: King W0=6 cluster of --n particles,
    the first --ni entries of its sorted step list; warm-up call, then one call."""
    import torch

    import workloads as W
    from paper_1504_03687_gb300 import Context
    dev = torch.device("cuda", 0)
    if args.model == "king":
        cl = W.king(args.n, 2, W0=6.0, masses="kroupa", binary_fraction=0.05)
    else:
        cl = W.plummer(args.n, 3, masses="kroupa")
    rs2 = W.neighbour_radius2(cl.x, 80, seed=2)
    order = W.sorted_step_list(W.block_steps(cl, seed=2)).astype(np.int32)
    a0, j0, tl = W.hermite_state(cl, seed=2, t_block=0.125)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    ctx = Context(cl.n, precision=args.prec, nb_cap=NB_CAP)
    ctx.set_particles(*[T(q) for q in (cl.x, cl.v, a0, j0, cl.m, tl)])
    idx = T(order[:args.ni])
    rs2_dev = torch.tensor([rs2], dtype=torch.float64, device=dev)
    rng = np.random.default_rng(0)
    g = [T(rng.standard_normal(s)) for s in ((args.ni, 3), (args.ni, 3), (args.ni,))]
    plans = [tuple(int(x) for x in v.split(":")) for v in args.variants.split(",") if v] or [None]
    ref = None
    for plan in plans:
        if plan is not None:
            ctx.set_plan_override(*plan)
        for it in range(2):
            ctx.set_timing(it == 1)
            ctx.predict(0.125)
            out = ctx.regular_force(idx, rs2_dev, neighbours=not args.no_lists,
                                    nb_capacity=0 if args.no_lists else args.ni * NB_PER_ROW)
            if args.backward:
                ctx.regular_force_backward(idx, *g)
            if args.irregular:
                ctx.irregular_force(0.125, idx, out.nb_off, out.nb_idx)
            ctx.sync()
        ph = ctx.timings()
        pairs = args.ni * cl.n
        res = {"case": f"{args.model} n={cl.n} n_i={args.ni} {args.prec}", "plan": ctx.plan(cl.n, args.ni),
               "phase_ms": {k: v[0] for k, v in ph.items()}, "launches": {k: v[1] for k, v in ph.items()},
               "force_Ginteractions_s": pairs / (ph["force"][0] * 1e-3) / 1e9 if ph["force"][0] > 0 else None,
               "nb_total": 0 if args.no_lists else int(out.nb_off[-1].item())}
        if args.irregular and ph["irregular"][0] > 0:
            res["irregular_Gpairs_s"] = res["nb_total"] / (ph["irregular"][0] * 1e-3) / 1e9
        if args.backward and ph["force"][0] > 0:
            fwd = ph["force"][0] + ph["reduce"][0] + ph["neighbours"][0]
            res["backward_over_forward"] = ph["backward"][0] / fwd
        if ref is None:
            ref = (out.acc.clone(), None if args.no_lists else out.nb_off.clone())
        else:  # every plan must give the same answer (to FP32 rounding of the partial sums)
            res["max_rel_acc_diff_vs_first"] = float(((out.acc - ref[0]).norm(dim=1) / ref[0].norm(dim=1)).max())
            if not args.no_lists:
                res["same_neighbour_offsets"] = bool(torch.equal(out.nb_off, ref[1]))
        print(json.dumps(res))


def bench_small_blocks(ctx, n, order, rs2_dev, dev, sizes=(1, 16, 128, 1024), reps=20):
    """Small active blocks of the same 2^20 cluster: the force call is then a pass over the j-records
    (48 B per particle, mixed) rather than arithmetic.  L2 flushed before every step (the step's
    predictor then writes the records its force call reads); median of `reps` calls of the force
    kernel (library CUDA events) and of the whole step (predict + force + reduce + neighbours).
    Achieved GB/s counts the record bytes once per call."""
    import torch
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    peak = None
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            peak = float(json.load(fh).get("hbm_gbs"))
    except Exception:
        pass
    rec_bytes = ((n + 255) // 256 * 256) * 48
    res = {"record_bytes": rec_bytes, "hbm_peak_gbs": peak,
           "l2": "flushed (512 MB write) before every step; the step's predictor writes the records",
           "blocks": {}}
    for b in sizes:
        idx = torch.as_tensor(order[:b], device=dev)
        force, step, phases = [], [], []
        for it in range(reps + 3):
            flush.fill_(it & 0xff)
            torch.cuda.synchronize()
            ctx.timings()
            ctx.set_timing(True)
            ctx.predict(0.125)
            ctx.regular_force(idx, rs2_dev, nb_capacity=b * NB_PER_ROW)
            ph = ctx.timings()
            ctx.set_timing(False)
            if it >= 3:
                force.append(ph["force"][0])
                step.append(sum(v[0] for v in ph.values()))
                phases.append(ph)
        f = float(np.median(force))
        gbs = rec_bytes / (f * 1e-3) / 1e9
        # where the step goes: predictor, row order, force, and the reduction + CSR (one launch
        # for blocks of at most 8 rows, timed as the reduction)
        med = {k: float(np.median([p[k][0] for p in phases])) for k in ("predict", "order", "force")}
        med["reduce_and_csr"] = float(np.median([p["reduce"][0] + p["neighbours"][0] for p in phases]))
        res["blocks"][str(b)] = {"force_ms_median": f, "step_ms_median": float(np.median(step)),
                                 "phase_ms_median": med,
                                 "achieved_GBs": gbs, "frac_of_hbm_peak": gbs / peak if peak else None,
                                 "plan": ctx.plan(n, b)}
    ctx.sync()
    return res


def bench_irregular(ctx, ctx64, cl, hermite, order, idx_dev, outs, rs2, reps=3):
    """Irregular force (Sec. 3.2.2) of the 2^14, 2^17 and 2^20 blocks of the timed step over the
    neighbour lists that step produced (cap 512), each active particle and its neighbours
    predicted on load (neighbour-only prediction), in the mixed context and in an FP64 one;
    then 32 sampled rows of the 2^20 block against the oracle with the oracle's own lists."""
    import torch

    import oracle
    a0, j0, tl = hermite
    t = 0.125
    res = {"workload": "lists of the timed step (r_s for a median of 80, cap 512); i and its neighbours "
                       "predicted from the Hermite state on load", "blocks": {}}
    for q, b in enumerate(BLOCKS):
        if b < BLOCKS[1]:
            continue
        off, nb = outs[q].nb_off, outs[q].nb_idx
        pairs = int(off[-1].item())
        row = {"neighbour_pairs": pairs}
        for name, c in (("mixed", ctx), ("fp64", ctx64)):
            c.irregular_force(t, idx_dev[q], off, nb)
            c.sync()
            c.timings()
            c.set_timing(True)
            for _ in range(reps):
                c.irregular_force(t, idx_dev[q], off, nb)
            ph = c.timings()
            c.set_timing(False)
            ms = ph["irregular"][0] / reps
            row[name] = {"ms": ms, "Gpairs_s": pairs / (ms * 1e-3) / 1e9}
        row["mixed_over_fp64"] = row["fp64"]["ms"] / row["mixed"]["ms"]
        res["blocks"][str(b)] = row
    rng = np.random.default_rng(7)
    rows = order[:BLOCKS[-1]][np.sort(rng.choice(BLOCKS[-1], 32, replace=False))]
    xp, vp = oracle.predict(t, cl.x, cl.v, a0, j0, tl)
    _, _, _, cnt, lists = oracle.regular_force(xp, vp, cl.m, rows, rs2, cap=NB_CAP)
    off = np.zeros(rows.size + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    flat = np.concatenate(lists).astype(np.int32)
    ref = oracle.irregular_force(t, cl.x, cl.v, a0, j0, tl, cl.m, rows, off, flat)
    has = cnt > 0
    dev = idx_dev[0].device
    T = lambda a_: torch.as_tensor(np.ascontiguousarray(a_), device=dev)
    for name, c in (("mixed", ctx), ("fp64", ctx64)):
        got = c.irregular_force(t, T(rows), T(off), T(flat))
        c.sync()
        e = {}
        for k, (g, r) in enumerate(zip(got, ref)):
            g = g.cpu().numpy()[has]
            r = r[has]
            d = np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1) if g.ndim == 2 else np.abs(g - r) / np.abs(r)
            e[("acc", "jerk", "pot")[k]] = {"median": float(np.median(d)), "max": float(d.max())}
        res[f"error_vs_oracle_{name}_32_rows"] = e
    return res


def bench_scheduler(dev, cl, steps=512, parity_steps=16):
    """Block-step sorting list (Sec. 3.3.1) on the 2^20-particle King cluster: levels from the
    local dynamical time (steps 2^-12 .. 2^-3), `steps` block steps with seeded level requests
    (a stand-in for the step criterion), timed on the host clock around nb_sched_next +
    nb_sched_update (which synchronises).  The first `parity_steps` steps are replayed by the
    reference scheduler with the same requests and the lists compared."""
    import torch

    import workloads as W
    from oracle.sorting_list import SortingList
    from paper_1504_03687_gb300 import Scheduler
    lv = W.step_levels(W.block_steps(cl, seed=2, dt_min=0.5 ** 12, dt_max=0.5 ** 3))
    # parity: the first steps against the reference, with requests from the reference's state
    ref = SortingList(lv, level_min=3, level_max=12, tick_level=48)
    sch = Scheduler(lv, 3, 12, device=dev.index or 0)
    t_ref = 0.0
    for k in range(parity_steps):
        t0 = time.perf_counter()
        T, act = ref.next()
        want = W.level_requests(ref.level[ref.order[:act.size]], seed=9000 + k)
        ref.update(want)
        t_ref += time.perf_counter() - t0
        sch.next()
        sch.update(want, granted=False)
    lst, lev, _ = sch.get()
    parity = bool(np.array_equal(lst, ref.order) and np.array_equal(lev, ref.level))
    sch.close()
    # timing: requests made on the device from the current levels (torch), not timed
    sch = Scheduler(lv, 3, 12, device=dev.index or 0)
    lev_t = torch.as_tensor(lv, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    delta = torch.tensor([-1, 0, 0, 0, 1, 2], dtype=torch.int32, device=dev)
    t_sched, part_steps, sizes = 0.0, 0, []
    for k in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t, na = sch.next()
        t_sched += time.perf_counter() - t0
        idx = sch.active().clone()
        want = lev_t[idx] + delta[torch.randint(0, 6, (na,), device=dev, generator=gen)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        granted = sch.update(want)
        t_sched += time.perf_counter() - t0
        lev_t[idx] = granted
        part_steps += na
        sizes.append(na)
    sch.close()
    return {"workload": "King W0=6 N=2^20, levels 3..12 from the local dynamical time, requests level "
                        "-1/0/+1/+2 with probabilities 1/6, 1/2, 1/6, 1/6",
            "block_steps": steps, "particle_steps": part_steps,
            "active_min": int(min(sizes)), "active_median": float(np.median(sizes)), "active_max": int(max(sizes)),
            "gpu_ms_total": t_sched * 1e3, "us_per_block_step": t_sched * 1e6 / steps,
            "ns_per_particle_step": t_sched * 1e9 / part_steps,
            "reference_us_per_block_step_first_steps": t_ref * 1e6 / parity_steps,
            "parity_with_reference_first_steps": parity, "parity_steps": parity_steps}


def bench_ac(dev, n=65536, t_end=1.0 / 64, precisions=("mixed", "fp64"), reference=True):
    """Ahmad-Cohen block-step integration on the device (nb_ac_*): Plummer N = 65536 with
    Kroupa masses, r_s adapted towards 50 neighbours (cap 256), eta_irr 0.02, eta_reg 0.03,
    from t = 0 to t_end, in a mixed and an FP64 context; wall time on the host clock, particle
    steps per second, energy error (oracle energy before and after).  The same run by the
    reference AC integrator on the host cores is timed beside it."""
    import torch

    import oracle
    import workloads as W
    from paper_1504_03687_gb300 import ACIntegrator, Context
    cl = W.plummer(n, 104, masses="kroupa")
    rs2 = W.neighbour_radius2(cl.x, 50, seed=104)
    kw = dict(eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=t_end, nb_opt=50)
    E0 = sum(oracle.energy(cl.m, cl.x, cl.v))
    res = {"workload": f"Plummer N={n} Kroupa, r_s towards 50 neighbours (cap 256), eta_irr 0.02, eta_reg 0.03, "
                       f"t = 0 .. {t_end} (= dt_max: every particle ends at t_end)"}
    for prec in precisions:
        ctx = Context(n, precision=prec, nb_cap=256, device=dev.index or 0)
        ctx.apply_tuned(n)  # the autotuner's launch plans for this particle count, if any
        ac = ACIntegrator(ctx, cl.m, cl.x, cl.v, rs2, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ac.run(t_end, max_blocks=1000000)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        g = ac.get()
        e = (sum(oracle.energy(cl.m, g["x"], g["v"])) - E0) / abs(E0)
        res[prec] = {"wall_s": wall, "block_steps": st["blocks"], "irregular_steps": st["irregular_steps"],
                     "regular_steps": st["regular_steps"], "particle_steps_per_s": st["irregular_steps"] / wall,
                     "ms_per_block_step": wall * 1e3 / max(st["blocks"], 1),
                     "us_per_block_step": wall * 1e6 / max(st["blocks"], 1),
                     "device_driven_block_steps": st["device_blocks"], "energy_rel_error": e,
                     "all_synchronised": bool(np.all(g["t"] == t_end)), "median_neighbours": float(np.median(g["nb_count"]))}
        ac.close()
        ctx.close()
    if not reference:
        return res
    t0 = time.perf_counter()
    ox, ov, _, info = oracle.ac_run(cl.m, cl.x, cl.v, rs2, t_end, cap=256, **kw)
    wall = time.perf_counter() - t0
    res["reference_on_host"] = {"wall_s": wall, "cores": oracle.num_threads(), "block_steps": info["blocks"],
                                "irregular_steps": info["irregular_steps"], "regular_steps": info["regular_steps"],
                                "energy_rel_error": (sum(oracle.energy(cl.m, ox, ov)) - E0) / abs(E0)}
    res["mixed_speedup_over_reference"] = wall / res["mixed"]["wall_s"]
    res["king_1m"] = bench_ac_king_1m(dev)
    res["plummer_1k_hermite_t1"] = bench_hermite_drift(dev)
    return res


def bench_hermite_drift(dev):
    """Energy drift of the block-step Hermite integration of the 1024-body equal-mass Plummer
    sphere to t = 1 (eta = 0.02, eta_s = 0.01, dt_max = 1/8): the oracle's FP64 run beside the
    device's FP64 and mixed runs (the AC integrator with r_s covering everything)."""
    import ctypes

    import oracle
    import workloads as W
    from paper_1504_03687_gb300 import ACIntegrator, Context
    cl, _ = W.plummer_1k_equal()
    E0 = sum(oracle.energy(cl.m, cl.x, cl.v))
    xh, vh = cl.x.copy(), cl.v.copy()
    st = np.zeros(4)
    oracle._load().orc_hermite_run(cl.n, cl.m.ctypes.data, xh.ctypes.data, vh.ctypes.data, ctypes.c_double(1.0),
                                   ctypes.c_double(0.02), ctypes.c_double(0.01), ctypes.c_double(0.125),
                                   ctypes.c_double(0.0), ctypes.c_int64(0), st.ctypes.data)
    res = {"oracle_fp64": (sum(oracle.energy(cl.m, xh, vh)) - E0) / abs(E0), "block_steps_oracle": int(st[0])}
    for prec in ("fp64", "mixed"):
        ctx = Context(cl.n, precision=prec, nb_cap=cl.n, device=dev.index or 0)
        ac = ACIntegrator(ctx, cl.m, cl.x, cl.v, 1e300, eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=0.125,
                          nb_opt=0)
        s_ = ac.run(1.0, max_blocks=100000)
        g = ac.get()
        res[f"device_{prec}"] = (sum(oracle.energy(cl.m, g["x"], g["v"])) - E0) / abs(E0)
        res[f"block_steps_{prec}"] = s_["blocks"]
        ac.close()
        ctx.close()
    return res


def gpu_energy(dev, m, x, v):
    """K + W with W = 1/2 sum m pot from the mixed all-pairs potentials on the device."""
    import torch

    from paper_1504_03687_gb300 import Context
    n = m.shape[0]
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    ctx = Context(n, precision="mixed", nb_cap=1, device=dev.index or 0)
    ctx.set_predicted(T(x), T(v), T(m))
    r = ctx.regular_force(T(np.arange(n, dtype=np.int32)), 0.0, neighbours=False)
    ctx.sync()
    W_ = 0.5 * float((T(m) * r.pot).sum().item())
    ctx.close()
    return 0.5 * float((m[:, None] * v * v).sum()) + W_


def bench_ac_king_1m(dev, t_end=1.0 / 64, dt_max=None):
    """The Ahmad-Cohen integrator on the million-body King W0 = 6 cluster (5 % binaries as
    centre-of-mass particles), mixed precision, r_s towards 50 neighbours (cap 256), from
    t = 0 to t_end (maximum step dt_max, by default t_end); wall time, particle steps, energy
    error from the mixed all-pairs potentials before and after.  Context: the paper's 1M runs took about 800 s of wall time
    per N-body time unit on 16 nodes (32 K20X + 320 CPU cores)."""
    import torch

    import workloads as W
    from paper_1504_03687_gb300 import ACIntegrator, Context
    cl, _ = W.king_1m_binaries()
    rs2 = W.neighbour_radius2(cl.x, 50, seed=2)
    E0 = gpu_energy(dev, cl.m, cl.x, cl.v)
    ctx = Context(cl.n, precision="mixed", nb_cap=256, device=dev.index or 0)
    ctx.apply_tuned(cl.n)
    ac = ACIntegrator(ctx, cl.m, cl.x, cl.v, rs2, eta_irr=0.02, eta_reg=0.03, eta_s=0.01,
                      dt_max=t_end if dt_max is None else dt_max, nb_opt=50)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ac.run(t_end, max_blocks=2000000)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    g = ac.get()
    ac.close()
    ctx.close()
    E1 = gpu_energy(dev, cl.m, g["x"], g["v"])
    return {"workload": "King W0=6 N=2^20 (5% binary c.m.), Kroupa, r_s towards 50 neighbours (cap 256), "
                        f"mixed, t = 0 .. {t_end}", "wall_s": wall, "block_steps": st["blocks"],
            "irregular_steps": st["irregular_steps"], "regular_steps": st["regular_steps"],
            "particle_steps_per_s": st["irregular_steps"] / wall, "wall_s_per_nbody_time_unit": wall / t_end,
            "dt_max": t_end if dt_max is None else dt_max,
            "energy_rel_error": (E1 - E0) / abs(E0), "all_synchronised": bool(np.all(g["t"] == t_end)),
            "context": "paper: about 800 s per N-body time unit for 1M on 16 nodes, 32 K20X + 320 CPU cores "
                       "(no binaries); this run is short and starts with small steps (eta_s), so the per-unit "
                       "figure is an upper bound"}


def bench_ensemble(dev, steps=5, n_clusters=512):
    """512 independent Plummer clusters (N log-uniform in 256..32768, active fraction uniform
    in 1/64..1): the batched form (one persistent launch, tile chosen by the autotuner,
    replayed from a captured CUDA graph) against one nb_regular_force launch per cluster."""
    import torch

    import oracle
    import workloads as W
    from paper_1504_03687_gb300 import Context, tune
    e = W.ensemble(n_clusters=n_clusters, seed=4)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    n = int(e.cluster_off[-1])
    rows = int(e.active_off[-1])
    pairs = int(sum((e.active_off[c + 1] - e.active_off[c]) * (e.cluster_off[c + 1] - e.cluster_off[c])
                    for c in range(n_clusters)))
    ctx = Context(n, precision="mixed", nb_cap=NB_CAP, device=dev.index or 0)
    ctx.set_predicted(T(e.x), T(e.v), T(e.m))
    idx, rs2 = T(e.idx), T(e.rs2)
    best_v, _ = tune.tune_batched(ctx, e.cluster_off, e.active_off, idx, rs2, log=lambda *a: None)
    ctx.batch_plan(e.cluster_off, e.active_off, best_v)
    cap = rows * 128
    out = ctx.regular_force_batched(idx, rs2, nb_capacity=cap)
    ctx.sync()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            ctx.regular_force_batched(idx, rs2, out=out)
    torch.cuda.current_stream(dev).wait_stream(side)
    g.replay()
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(steps):
        g.replay()
    ev[1].record()
    torch.cuda.synchronize(dev)
    t_batched = ev[0].elapsed_time(ev[1]) / steps
    # baseline: one context per cluster, one nb_regular_force launch sequence per cluster
    ctxs = []
    for c in range(n_clusters):
        lo, hi = e.cluster_off[c], e.cluster_off[c + 1]
        cc = Context(int(hi - lo), precision="mixed", nb_cap=NB_CAP, device=dev.index or 0)
        cc.set_predicted(T(e.x[lo:hi]), T(e.v[lo:hi]), T(e.m[lo:hi]))
        li = T((e.idx[e.active_off[c]:e.active_off[c + 1]] - lo).astype(np.int32))
        r2 = T(e.rs2[c:c + 1])
        o = cc.regular_force(li, r2, nb_capacity=int(li.numel()) * 128)
        ctxs.append((cc, li, r2, o))
    torch.cuda.synchronize(dev)
    ev[0].record()
    for _ in range(steps):
        for cc, li, r2, o in ctxs:
            cc.regular_force(li, r2, out=o)
    ev[1].record()
    torch.cuda.synchronize(dev)
    t_single = ev[0].elapsed_time(ev[1]) / steps
    # accuracy of the batched result on 8 sampled clusters
    acc = out.acc.cpu().numpy()
    errs = []
    for c in np.random.default_rng(0).choice(n_clusters, 8, replace=False):
        lo, hi = e.cluster_off[c], e.cluster_off[c + 1]
        r0, r1 = e.active_off[c], e.active_off[c + 1]
        ref = oracle.regular_force(e.x[lo:hi], e.v[lo:hi], e.m[lo:hi], (e.idx[r0:r1] - lo).astype(np.int32),
                                   e.rs2[c], cap=NB_CAP, lists=False)
        errs.append(np.linalg.norm(acc[r0:r1] - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1))
    errs = np.concatenate(errs)
    for cc, *_ in ctxs:
        cc.close()
    ctx.close()
    return {"workload": f"{n_clusters} Plummer clusters, N log-uniform 256..32768 (sum {n}), active fraction "
                        f"U(1/64,1) ({rows} rows), equal masses, r_s for 50 neighbours",
            "pairs": pairs, "batched_variant": int(best_v),
            "batched_graph_ms": t_batched, "batched_Ginteractions_s": pairs / (t_batched * 1e-3) / 1e9,
            "per_cluster_ms": t_single, "per_cluster_Ginteractions_s": pairs / (t_single * 1e-3) / 1e9,
            "speedup": t_single / t_batched,
            "acc_error_vs_oracle_8_clusters": {"median": float(np.median(errs)), "max": float(errs.max())}}


def bench_adjoint(dev, reps=3):
    """Adjoint of force+jerk+potential at N = 65536 (Plummer, Kroupa), full active block, for
    L = sum(w.acc + u.jerk) + sum(pot) with w, u ~ N(0,1): forward vs backward device time,
    and the GPU gradient against O(N) central differences of the FP64 oracle at 64 random
    coordinates of x, v and m.  Then the gradient of the final kinetic energy through 64
    block steps at N = 16384 with checkpoint-and-recompute every 8 steps (mixed and FP64)."""
    import torch

    import oracle
    import workloads as W
    from paper_1504_03687_gb300 import Context
    from paper_1504_03687_gb300.autograd import hermite_chain
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    cl, _ = W.plummer_64k_kroupa()
    n = cl.n
    rng = np.random.default_rng(3)
    ga, gj, gp = rng.standard_normal((n, 3)), rng.standard_normal((n, 3)), np.ones(n)
    idx = np.arange(n, dtype=np.int32)
    picks = [(["x", "v", "m"][q % 3], int(rng.integers(0, n)), int(rng.integers(0, 3))) for q in range(64)]
    fd = np.array([oracle.loss_fd(cl.x, cl.v, cl.m, idx, ga, gj, gp, w, p, c,
                                  h=1e-6 if w != "m" else 1e-6 * cl.m[p]) for w, p, c in picks])
    res = {}
    for prec in ("mixed", "fp64"):
        ctx = Context(n, precision=prec, nb_cap=64, device=dev.index or 0)
        ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
        idx_t, g = T(idx), [T(ga), T(gj), T(gp)]
        ctx.regular_force(idx_t, 0.0, neighbours=False)
        gx, gv, gm = ctx.regular_force_backward(idx_t, *g)
        ctx.sync()
        ctx.timings()
        ctx.set_timing(True)
        for _ in range(reps):
            ctx.regular_force(idx_t, 0.0, neighbours=False)
        for _ in range(reps):
            gx, gv, gm = ctx.regular_force_backward(idx_t, *g)
        ph = ctx.timings()
        ctx.set_timing(False)
        fwd = (ph["force"][0] + ph["reduce"][0]) / reps
        bwd = ph["backward"][0] / reps
        gx, gv, gm = gx.cpu().numpy(), gv.cpu().numpy(), gm.cpu().numpy()
        got = np.array([gx[p, c] if w == "x" else gv[p, c] if w == "v" else gm[p] for w, p, c in picks])
        scale = np.array([np.abs(gx).max() if w == "x" else np.abs(gv).max() if w == "v" else np.abs(gm).max()
                          for w, _, _ in picks])
        err = np.abs(got - fd) / np.maximum(np.abs(fd), 1e-4 * scale)
        res[prec] = {"forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
                     "backward_Gpairs_s": 2 * n * n / (bwd * 1e-3) / 1e9,
                     "fd_rel_err_64_coords": {"median": float(np.median(err)), "max": float(err.max())}}
        ctx.close()
    # gradient through K block steps of a frozen schedule, checkpoint every 8
    cl2 = W.plummer(16384, 33, masses="kroupa")
    K = 64
    _, _, sched = oracle.hermite_record(cl2.m, cl2.x, cl2.v, 1.0, eta=0.02, max_blocks=K)
    chain = {"n": cl2.n, "block_steps": len(sched), "particle_steps": int(sum(len(a) for _, a in sched))}
    for prec in ("mixed", "fp64"):
        ctx = Context(cl2.n, precision=prec, nb_cap=64, device=dev.index or 0)
        schedule = [(t, T(a)) for t, a in sched]
        times = []
        for it in range(2):
            x0 = T(cl2.x).requires_grad_(True)
            v0 = T(cl2.v).requires_grad_(True)
            m = T(cl2.m)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            xf, vf = hermite_chain(x0, v0, m, schedule, ctx, checkpoint_every=8)
            ke = 0.5 * (m[:, None] * vf * vf).sum()
            ke.backward()
            torch.cuda.synchronize(dev)
            times.append(time.perf_counter() - t0)
        chain[prec] = {"forward_plus_backward_s": times[-1], "final_kinetic_energy": float(ke.item()),
                       "grad_norm_x0": float(x0.grad.norm().item()), "grad_norm_v0": float(v0.grad.norm().item())}
        ctx.close()
    res["hermite_chain_K64_N16384"] = chain
    return res


def host_force(ctx, idx, rs2, out):
    """nb_regular_force with host buffers; returns the bytes copied device->host."""
    import ctypes
    lib = ctx.lib
    n_i = idx.shape[0]
    rs2a = np.array([rs2], dtype=np.float64)
    s = lib.nb_regular_force(ctx.h, n_i, idx.ctypes.data, rs2a.ctypes.data, 1, out.acc.ctypes.data,
                             out.jerk.ctypes.data, out.pot.ctypes.data, out.nb_off.ctypes.data,
                             out.nb_idx.ctypes.data, out.nb_idx.shape[0], out.nb_count.ctypes.data, 0)
    if s not in (0, 5):
        raise RuntimeError(f"nb_regular_force failed: {s} {lib.nb_last_error(ctx.h).decode()}")
    used = int(min(out.nb_off[-1], out.nb_idx.shape[0]))
    return n_i * (24 + 24 + 8 + 4) + (n_i + 1) * 8 + used * 4


if __name__ == "__main__":
    main()
