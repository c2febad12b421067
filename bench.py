#!/usr/bin/env python3
"""Throughput of the Shield-MPPI hot path on GB300.

The unit of work is one whole Shield-MPPI control update (Alg. 2 body) of the
K = 65536, T = 100 problem (elliptical 20 x 12 m track, half-width 2 m): K
sampled rollouts with the DCBF cost and the softmin update, up to 10 Armijo
repair iterations of V+ (they run while V+ breaks the DCBF condition), then
the disturbed closed-loop step and warm start, all through
smppi_shield_update.  One timed step is R such updates back to back (R chosen
so that the timed region lasts over a second), each bracketed by CUDA events
with the L2 flushed before it.  The metric is rollout-steps/s = K T / (time
per update); the line also carries the microseconds per update, the repair
iterations that ran, a second workload whose near-boundary starts make the
shield iterate, the roofline of the dominant kernel, the end-to-end rate
through the host-buffer API and the FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank runs its own problem
instance (an independent Philox stream): weak scaling, no collective on the
data path; rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rollout-steps/s & µs per MPPI update (batched+adjoint vs plain), % FP32 roofline"
UNIT = "rollout-steps/s"
K_ROLL, T_HOR, N_REPAIR = 65536, 100, 10
# FP32 flops of one rollout step (FMA = 2), hand count: Box-Muller pair and
# uniforms 44, perturbation and control-cost term 10, two slip angles 48, two
# lateral forces 34, steer sin/cos 28, force balance 20, heading increment 32,
# Euler update 12, track projection (about three segments) 39, running cost and
# DCBF penalty 13.
F_ALG = 280
# FP32 peak: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
L2_FLUSH_BYTES = 256 << 20
# DRAM traffic per rollout launch from the ncu capture in profiles/, valid only
# for the kernel source it was taken on (hash of the files that define it).
ROLLOUT_TRAFFIC = {"sources_sha": "69b15b31bd555004", "bytes_per_launch": 139776}


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("rollout.cu", "rollout2.cuh", "device.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2302_11719_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while timing runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and all(v.strip().isdigit() for v in ids):
        return int(ids[local_rank % len(ids)])
    return local_rank


# --------------------------------------------------------------------------
def oracle_updates(K, T, n_repair, budget_s, nthreads, max_updates=None):
    """Time whole Shield-MPPI updates of the FP64 oracle (closed loop) on the host."""
    import numpy as np

    import oracle as O
    from paper_2302_11719_gb300 import inputs as I
    O.build()
    pr = I.throughput_problem(K, T)
    m = O.Model(pr.params, pr.track)
    x0 = pr.x0.astype(np.float64)
    V = pr.V.astype(np.float64)
    n, t0 = 0, time.perf_counter()
    times = []
    while True:
        a = time.perf_counter()
        _, Vp = O.mppi_step(m, x0, V, n, 0, nthreads=nthreads)
        Vs, _, _, _ = O.repair(m, x0, Vp, n_repair)
        x0 = O.apply(m, x0, Vs[0], n)
        V = O.shift(m, Vp)
        times.append(time.perf_counter() - a)
        n += 1
        if (max_updates and n >= max_updates) or (not max_updates and
                                                   time.perf_counter() - t0 > budget_s):
            break
    return n, times


def oracle_problem_updates(pr, n_repair, n_updates, nthreads):
    """Time closed-loop updates of the FP64 oracle on the host for problem pr
    (the CPU-baseline leg of the small configurations)."""
    import numpy as np

    import oracle as O
    O.build()
    m = O.Model(pr.params, pr.track)
    x0 = pr.x0.astype(np.float64)
    V = pr.V.astype(np.float64)
    times = []
    for n in range(n_updates):
        a = time.perf_counter()
        _, Vp = O.mppi_step(m, x0, V, n, 0, nthreads=nthreads)
        Vs = Vp
        if n_repair > 0:
            Vs, _, _, _ = O.repair(m, x0, Vp, n_repair)
        x0 = O.apply(m, x0, Vs[0], n)
        V = O.shift(m, Vp)
        times.append(time.perf_counter() - a)
    return times


def cpu_threads() -> int:
    return os.cpu_count() or 1


def run_reference(args):
    _, rank, _ = dist_env()
    if rank != 0:
        return 0
    nth = cpu_threads()
    # warm-up updates, then the timed ones (full-size updates of the oracle)
    oracle_updates(K_ROLL, T_HOR, N_REPAIR, 0, nth, max_updates=max(1, args.warmup))
    n, times = oracle_updates(K_ROLL, T_HOR, N_REPAIR, 0, nth, max_updates=args.steps)
    total = sum(times)
    value = K_ROLL * T_HOR * n / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": n, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / n, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nth, "kind": "oracle",
                         "sample": "%d whole Shield-MPPI updates (K=%d, T=%d, %d repair "
                                   "iterations) of the FP64 oracle" % (n, K_ROLL, T_HOR,
                                                                      N_REPAIR)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(updates_per_step=1):
    return {"workload": "Shield-MPPI control update, K=%d rollouts, T=%d, up to %d Armijo repair "
                        "iterations (they run only while V+ breaks the DCBF condition), closed "
                        "loop" % (K_ROLL, T_HOR, N_REPAIR),
            "K": K_ROLL, "T": T_HOR, "n_repair_max": N_REPAIR,
            "updates_per_step": updates_per_step,
            "track": "ellipse 20 x 12 m, half-width 2 m, 1024 points",
            "model": "6-state dynamic single-track car, dt 0.02 s",
            "l2": "flushed before every timed update (256 MiB write, outside the timed events)"}


def updates_per_step(steps, est_update_s, min_timed_s):
    """Updates per timed step so that steps x R updates last at least min_timed_s."""
    return max(1, int(math.ceil(min_timed_s / (steps * max(est_update_s, 1e-6)))))


def iterations_run(merit_row, n_repair):
    """Repair iterations one update ran, from its merit row (P before each
    iteration and after the last, repeated after an early stop: a safe V,
    P = 0, or a line search that accepted nothing)."""
    for i in range(n_repair):
        if merit_row[i] == 0.0 or merit_row[i + 1] == merit_row[i]:
            return i
    return n_repair


def shield_active_workload(S, I, dev, flush, n_updates, inst):
    """Updates in which the shield works: each starts from a near-boundary state
    (offset 1.5-1.95 m of the 2 m half-width, heading 0.1 rad outward) with a
    warm start that steers further out (inputs.near_boundary_sequences), so V+
    often breaks the DCBF condition and the Armijo repair iterates.  Same K, T
    and track as the headline; every update is timed with its own events."""
    import numpy as np
    import torch
    sb = I.near_boundary_sequences(n_updates, T_HOR, seed=1)
    pr = I.throughput_problem(K_ROLL, T_HOR)
    ctl = S.Controller(pr.params, pr.track, device=dev)
    xs, Vs_all = ctl.tensor(sb.x0), ctl.tensor(sb.V)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    Vs = torch.empty_like(V)
    merits = torch.zeros((n_updates, N_REPAIR + 1), dtype=torch.float64, device=dev)
    for j in range(3):                                  # warm-up
        x0.copy_(xs[j]); V.copy_(Vs_all[j])
        S.smppi_shield_update(ctl.h, x0, V, Vs, j, inst, N_REPAIR)
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(n_updates)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(n_updates)]
    for j in range(n_updates):
        x0.copy_(xs[j]); V.copy_(Vs_all[j])
        flush.zero_()
        e0[j].record()
        S.smppi_shield_update(ctl.h, x0, V, Vs, 100 + j, inst, N_REPAIR, merits[j])
        e1[j].record()
    torch.cuda.synchronize()
    st, bits = ctl.sync_status()
    ms = np.array([a.elapsed_time(b) for a, b in zip(e0, e1)])
    mer = merits.cpu().numpy()
    it = np.array([iterations_run(r, N_REPAIR) for r in mer])
    ctl.close()
    rep = it > 0
    return {"workload": "near-boundary starts (offset 1.5-1.95 m, heading 0.1 rad outward, warm "
                        "start steering outward), K=%d, T=%d, up to %d Armijo iterations"
                        % (K_ROLL, T_HOR, N_REPAIR),
            "updates": n_updates, "us_per_update": 1e3 * float(ms.mean()),
            "us_per_update_with_repair": 1e3 * float(ms[rep].mean()) if rep.any() else None,
            "us_per_update_without_repair": 1e3 * float(ms[~rep].mean()) if (~rep).any() else None,
            "repair_iterations_run_mean": float(it.mean()),
            "updates_with_repair": int(rep.sum()),
            "merit_before_mean": float(mer[:, 0].mean()),
            "merit_after_mean": float(mer[:, -1].mean()),
            "safe_after": int((mer[:, -1] == 0.0).sum()),
            "status_bits": int(bits)}


def dist_env():
    """(world size, rank, local rank) from the torchrun environment; (1, 0, 0) without it."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself when there is no process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, max_seconds):
    """Whole-job throughput under weak scaling: every rank runs its own problem of
    the same size (replicas; rank r uses Philox instance r), so the job processed
    world x units_per_rank in the slowest rank's time."""
    return world * units_per_rank / max_seconds


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2302_11719_gb300 import inputs as I
    from paper_2302_11719_gb300 import smppi as S

    world, rank, local = dist_env()
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    pr = I.throughput_problem(K_ROLL, T_HOR)
    ctl = S.Controller(pr.params, pr.track, device=dev)
    inst = rank
    x0 = ctl.tensor(pr.x0)
    V = ctl.tensor(pr.V)
    Vs = torch.empty_like(V)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    it = 0
    wu0 = time.perf_counter()
    for _ in range(args.warmup):
        S.smppi_shield_update(ctl.h, x0, V, Vs, it, inst, N_REPAIR)
        it += 1
    torch.cuda.synchronize()
    est_s = (time.perf_counter() - wu0) / args.warmup
    st, bits = ctl.sync_status()
    if st not in (S.OK, S.ERR_STALLED):
        raise RuntimeError("device status %d (bits %d) in warm-up" % (st, bits))

    # one step = R back-to-back control updates (R chosen so that the timed
    # region lasts at least --min-timed-seconds; each update is bracketed by its
    # own events with the L2 flush before it, outside the events)
    R = updates_per_step(args.steps, est_s, args.min_timed_seconds)
    n_upd = args.steps * R
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(n_upd)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(n_upd)]
    merits = torch.zeros((n_upd, N_REPAIR + 1), dtype=torch.float64, device=dev)
    sampler = ClockSampler(gpu_index(local))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    wall0 = time.perf_counter()
    for j in range(n_upd):
        flush.zero_()
        e0[j].record()
        S.smppi_shield_update(ctl.h, x0, V, Vs, it, inst, N_REPAIR, merits[j])
        e1[j].record()
        it += 1
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    upd_ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    step_ms = [sum(upd_ms[i * R:(i + 1) * R]) for i in range(args.steps)]
    iters = [iterations_run(row, N_REPAIR) for row in merits.cpu().numpy()]
    # per-kernel durations: the same steps again with CUDA events around every
    # launch (on the library's stream).  Events between the launches cost time
    # and stop a launch from overlapping its predecessor's tail, so the step
    # times above are taken without them.
    S.smppi_timing(ctl.h, True)
    for i in range(args.steps):
        flush.zero_()
        S.smppi_shield_update(ctl.h, x0, V, Vs, it, inst, N_REPAIR)
        it += 1
    torch.cuda.synchronize()
    S.smppi_timing(ctl.h, False)
    # context: the same updates chained as a control loop runs them (one L2 flush
    # and one event pair per group of R updates; the next update's rollout
    # launch becomes resident while the previous shield runs)
    b2b_ms = []
    for i in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(R):
            S.smppi_shield_update(ctl.h, x0, V, Vs, it, inst, N_REPAIR)
            it += 1
        b.record()
        b2b_ms.append((a, b))
    torch.cuda.synchronize()
    b2b_us = 1e3 * statistics.median(a.elapsed_time(b) for a, b in b2b_ms) / R
    clocks = sampler.stop()
    kt = S.smppi_timing_read(ctl.h)
    total_s = sum(step_ms) / 1e3
    st, bits = ctl.sync_status()
    if st not in (S.OK, S.ERR_STALLED):
        raise RuntimeError("device status %d (bits %d) in the timed region" % (st, bits))
    total_s = max_over_ranks(total_s, dist, dev)
    value = job_rate(world, K_ROLL * T_HOR * n_upd, total_s)

    # end to end through the host-buffer entry point (copies in the timed region)
    hx = torch.from_numpy(pr.x0.copy()).pin_memory()
    hV = torch.from_numpy(pr.V.copy()).pin_memory()
    hVs = torch.empty_like(hV).pin_memory()
    for _ in range(2):
        S.smppi_shield_update(ctl.h, hx.data_ptr(), hV.data_ptr(), hVs.data_ptr(), it, inst,
                              N_REPAIR, None, True)
        it += 1
    e2e_s = 0.0
    for i in range(n_upd):
        flush.zero_()
        torch.cuda.synchronize()
        a = time.perf_counter()
        S.smppi_shield_update(ctl.h, hx.data_ptr(), hV.data_ptr(), hVs.data_ptr(), it, inst,
                              N_REPAIR, None, True)
        e2e_s += time.perf_counter() - a
        it += 1
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_value = job_rate(world, K_ROLL * T_HOR * n_upd, e2e_s)
    active = shield_active_workload(S, I, dev, flush, args.active_updates, inst)

    if rank != 0:
        dist.barrier()
        dist.destroy_process_group()
        ctl.close()
        return 0

    # roofline of the dominant kernel (largest share of the timed kernel time)
    shares = {k: v[0] for k, v in kt.items() if v[1] > 0}
    tot_k = sum(shares.values())
    dominant = max(shares, key=shares.get)
    roll_ms, roll_n = kt["rollout"]
    roll_avg_s = roll_ms / roll_n / 1e3
    achieved = F_ALG * K_ROLL * T_HOR / roll_avg_s / 1e12
    sha = kernel_sha()
    traffic = (ROLLOUT_TRAFFIC["bytes_per_launch"]
               if ROLLOUT_TRAFFIC["sources_sha"] == sha else None)
    roofline = {"bound": "alu", "kernel": "rollout", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                "flops_per_unit": F_ALG, "units_per_launch": K_ROLL * T_HOR,
                "avg_launch_us": roll_avg_s * 1e6}
    n_cpu = cpu_threads()
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        n, times = oracle_updates(K_ROLL, T_HOR, N_REPAIR, args.cpu_seconds, n_cpu)
        cpu = {"value": K_ROLL * T_HOR * n / sum(times), "unit": UNIT, "cores": n_cpu,
               "kind": "oracle",
               "sample": "%d whole Shield-MPPI updates (K=%d, T=%d, %d repair iterations) of "
                         "the FP64 oracle, %.1f s" % (n, K_ROLL, T_HOR, N_REPAIR, sum(times))}
    launches = 2 * n_upd        # rollout + update/shield launch per update in the timed region
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload_config(R),
        "updates_per_step": R,
        "us_per_update": 1e6 * total_s / n_upd,
        "update_us_median": 1e3 * statistics.median(upd_ms),
        "back_to_back": {"us_per_update": b2b_us,
                         "l2": "flushed before each group of %d chained updates" % R,
                         "note": "context only; the headline value flushes L2 before every update"},
        "step_ms_median": statistics.median(step_ms),
        "wall_s_timed_loop": wall,
        "repair_iterations_run": {"mean": float(np.mean(iters)), "max": int(max(iters)),
                                  "updates_with_repair": int(sum(i > 0 for i in iters)),
                                  "updates": n_upd},
        "shield_active": active,
        "kernel_share": {k: round(v / tot_k, 4) for k, v in shares.items()},
        "kernel_avg_us": {k: 1e3 * v[0] / v[1] for k, v in kt.items() if v[1]},
        "kernel_timing": "CUDA events around every launch on the library stream, in a second "
                         "pass of the same number of steps (L2 flushed between steps)",
        "dominant_kernel": dominant,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * (6 + 2 * T_HOR),
                "d2h_bytes_per_step": 4 * (6 + 4 * T_HOR)},
        "gpu_launches": launches,
        "gpu_launches_kernel_pass": sum(v[1] for v in kt.values()),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctl.close()
    return 0


def run_sharded(args):
    """--shard-rollouts: the ranks split the K rollouts of ONE problem (strong
    scaling).  Each update: every rank runs its slice (smppi_step_partial, the
    slice's Philox counters), one all-gather of the (2T + 2)-value partials
    over NCCL, the merge into V+ on every rank (smppi_merge_partials), then the
    shield and the closed-loop step, replicated (smppi_repair, smppi_apply)."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2302_11719_gb300 import inputs as I
    from paper_2302_11719_gb300 import smppi as S

    world, rank, local = dist_env()
    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pr = I.throughput_problem(K_ROLL, T_HOR)
    ctl = S.Controller(pr.params, pr.track, device=dev)
    k_lo, k_hi = S.shard_range(K_ROLL, world, rank)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    Vs = torch.empty_like(V)
    W = 2 * T_HOR + 2
    mine = torch.empty(W, dtype=torch.float64, device=dev)
    parts = torch.empty((world, W), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def update(it):
        S.smppi_step_partial(ctl.h, x0, V, it, 0, k_lo, k_hi, mine)
        if dist:
            dist.all_gather_into_tensor(parts, mine)
        else:
            parts[0].copy_(mine)
        S.smppi_merge_partials(ctl.h, world, parts, V)
        S.smppi_repair(ctl.h, 1, x0, V, Vs, N_REPAIR, 1)
        S.smppi_apply(ctl.h, x0, V, Vs, it, 0)

    for it in range(args.warmup):
        update(it)
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        e0[i].record()
        update(args.warmup + i)
        e1[i].record()
    torch.cuda.synchronize()
    st, bits = ctl.sync_status()
    if st not in (S.OK, S.ERR_STALLED):
        raise RuntimeError("device status %d (bits %d)" % (st, bits))
    total_s = sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / 1e3
    total_s = max_over_ranks(total_s, dist, dev)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": K_ROLL * T_HOR * args.steps / total_s, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(), parallelism="rollouts sharded over %d ranks, "
                           "all-gather of the slice partials" % world),
            "rollouts_per_rank": k_hi - k_lo,
            "gpu_launches": 6 * args.steps}), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctl.close()
    return 0


def _timed_steps(fn, steps, flush):
    """Per-step CUDA-event times (ms) of fn(i), L2 flushed before each step."""
    import torch
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        e0[i].record()
        fn(i)
        e1[i].record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(e0, e1)]


def _status_names(bits):
    """Names of the device status bits: 'stalled' means that in some update of
    some problem the repair line search accepted no step (the update then
    applies the last accepted iterate); it is not an error."""
    names = [n for b, n in ((1, "numeric"), (2, "timeout"), (4, "stalled")) if bits & b]
    return names or ["ok"]


def run_batch(args):
    """512 uneven Shield-MPPI problems: one persistent launch per closed-loop
    update vs 512 separate per-problem updates on one stream."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2302_11719_gb300 import inputs as I
    from paper_2302_11719_gb300 import smppi as S
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ib = I.uneven_instances(512, seed=0)
    B, n_rep = len(ib.params), N_REPAIR
    bt = S.Batch(ib, block_rollouts=0, device=dev)
    it = 0
    for _ in range(args.warmup):
        S.smppi_batch_step(bt.b, bt.x0, bt.V, bt.V_safe, it, n_rep)
        it += 1
    S.smppi_batch_sync_status(bt.b)
    rb, grid = S.smppi_batch_config(bt.b)

    def batched(i):
        S.smppi_batch_step(bt.b, bt.x0, bt.V, bt.V_safe, it + i, n_rep)
    t_b = _timed_steps(batched, args.steps, flush)
    it += args.steps
    # graph replays of the whole closed loop (no flush between replays)
    n_loop = args.loop_updates or 500
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    S.smppi_batch_loop(bt.b, bt.x0, bt.V, bt.V_safe, it, n_rep, 1)
    torch.cuda.synchronize()
    a0.record()
    S.smppi_batch_loop(bt.b, bt.x0, bt.V, bt.V_safe, it, n_rep, n_loop)
    a1.record()
    torch.cuda.synchronize()
    t_loop = a0.elapsed_time(a1)
    st_b = S.smppi_batch_sync_status(bt.b)
    # the same problems as 512 separate per-problem updates (handle path)
    ctls, states = [], []
    for i in range(B):
        c = S.Controller(ib.params[i], ib.tracks[i], device=dev)
        ctls.append(c)
        states.append((c.tensor(ib.x0[i]), c.tensor(np.zeros((c.T, 2), np.float32)),
                       torch.empty((c.T, 2), device=dev)))

    def plain(i):
        for j in range(B):
            x0, V, Vs = states[j]
            S.smppi_shield_update(ctls[j].h, x0, V, Vs, i, j, n_rep)
    for w in range(2):
        plain(w)
    torch.cuda.synchronize()
    t_p = _timed_steps(lambda i: plain(100 + i), max(3, args.steps // 4), flush)
    for c in ctls:
        c.close()
    rs_b = sum(int(k) * int(t) for k, t in zip(ib.K, ib.T))
    line = {
        "workload": "batched Shield-MPPI, 512 problems, K log-uniform [64, 16384], T in [20, 150], "
                    "ellipses 10-40 m, w in [1.5, 3] m, %d repair iterations, closed loop" % n_rep,
        "metric": "control updates/s", "unit": "updates/s",
        "batched": {"value": B * args.steps / (sum(t_b) / 1e3), "ms_per_update_all": float(np.median(t_b)),
                    "rollout_steps_per_s": rs_b * args.steps / (sum(t_b) / 1e3),
                    "block_rollouts": rb, "grid": grid, "l2": "flushed between steps"},
        "batched_graph_loop": {"value": B * n_loop / (t_loop / 1e3), "updates": n_loop,
                               "ms_per_update_all": t_loop / n_loop, "l2": "not flushed",
                               "device_status_bits": _status_names(st_b[1])},
        "plain_per_problem": {"value": B * len(t_p) / (sum(t_p) / 1e3),
                              "ms_per_update_all": float(np.median(t_p)),
                              "launches_per_update": 2 * B, "l2": "flushed between steps"},
        "speedup": (B * args.steps / (sum(t_b) / 1e3)) / (B * len(t_p) / (sum(t_p) / 1e3)),
    }
    print(json.dumps(line), flush=True)
    bt.close()
    return 0


def run_sweep(args):
    """One MPPI iteration (rollouts + update) for K x T on the single-problem workload."""
    import torch

    import __graft_entry__
    from paper_2302_11719_gb300 import inputs as I
    from paper_2302_11719_gb300 import smppi as S
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rows = []
    for K in (4096, 16384, 65536, 262144):
        for T in (50, 100, 200):
            pr = I.throughput_problem(K, T)
            ctl = S.Controller(pr.params, pr.track, device=dev)
            x0, V0 = ctl.tensor(pr.x0), ctl.tensor(pr.V)
            n_b = args.warmup + 2 * args.steps
            Vb = [V0.clone() for _ in range(n_b)]
            for i in range(args.warmup):
                S.smppi_step(ctl.h, x0, Vb[i], i, 0)
            t = _timed_steps(lambda i: S.smppi_step(ctl.h, x0, Vb[args.warmup + i], i, 0),
                             args.steps, flush)
            # per-kernel durations from a second pass with events around the launches
            S.smppi_timing(ctl.h, True)
            _timed_steps(lambda i: S.smppi_step(ctl.h, x0, Vb[args.warmup + args.steps + i], i, 0),
                         args.steps, flush)
            S.smppi_timing(ctl.h, False)
            kt = S.smppi_timing_read(ctl.h)
            roll_s = kt["rollout"][0] / kt["rollout"][1] / 1e3
            upd_s = kt["update"][0] / kt["update"][1] / 1e3
            step_s = sum(t) / len(t) / 1e3
            ach = F_ALG * K * T / roll_s / 1e12
            rows.append({"K": K, "T": T, "us_per_update": step_s * 1e6,
                         "rollout_steps_per_s": K * T / step_s,
                         "rollout_kernel_us": roll_s * 1e6, "update_kernel_us": upd_s * 1e6,
                         "fp32_tflops": ach, "fp32_frac": ach / FP32_PEAK_TFLOPS})
            ctl.close()
    # the FP64 oracle's MPPI iteration at K = 4096 and 65536, T = 100 (host cores)
    import numpy as np

    import oracle as O
    O.build()
    oracle_rows = []
    for K in (4096, 65536):
        pr = I.throughput_problem(K, 100)
        m = O.Model(pr.params, pr.track)
        x0, V = pr.x0.astype(np.float64), pr.V.astype(np.float64)
        for nth in (1, cpu_threads()):
            reps = 1 if (nth == 1 and K > 4096) else 3
            t = []
            for r in range(reps):
                a = time.perf_counter()
                O.mppi_step(m, x0, V, r, 0, nthreads=nth)
                t.append(time.perf_counter() - a)
            us = 1e6 * sum(t) / len(t)
            oracle_rows.append({"K": K, "T": 100, "threads": nth, "us_per_update": us,
                                "rollout_steps_per_s": K * 100 / (us * 1e-6)})
    print(json.dumps({"workload": "MPPI iteration sweep (rollouts + softmin update)",
                      "peak_tflops": FP32_PEAK_TFLOPS, "flops_per_rollout_step": F_ALG,
                      "l2": "flushed between steps", "rows": rows,
                      "oracle_fp64_host": oracle_rows}), flush=True)
    return 0


# The same count for the curvilinear model: noise 44, perturbation 10, slip angles
# 48, lateral forces 34, steer sin/cos 28, force balance 20, curvature lookup 8,
# 1 - kappa e_y and its reciprocal 4, s' e_y' e_psi' 10, heading rotation 27,
# Euler update 10, cost and DCBF penalty 17.
F_ALG_CURV = 260


def _time_repairs(S, ctl, n, x0, V, n_iters, args, flush):
    """smppi_repair of n sequences, n_iters iterations, in modes 1 (projected
    gradient + Armijo) and 2 (BFGS): time per call and what the repair achieved."""
    import torch
    dev = x0.device
    Vout = torch.empty_like(V)
    its = torch.empty(n, dtype=torch.int32, device=dev)
    mer = torch.empty((n, n_iters + 1), dtype=torch.float64, device=dev)
    out = {}
    for key, mode in (("repair_%d" % n_iters, 1), ("bfgs_%d" % n_iters, 2)):
        for _ in range(2):
            S.smppi_repair(ctl.h, n, x0, V, Vout, n_iters, mode, 0.0, mer, its)
        t = _timed_steps(lambda i: S.smppi_repair(ctl.h, n, x0, V, Vout, n_iters, mode, 0.0, mer,
                                                  its),
                         max(3, args.steps // 4), flush)
        st, bits = ctl.sync_status()
        iters = its.cpu().numpy()
        m = mer.cpu().numpy()
        us = 1e3 * sum(t) / len(t)
        out[key] = {"us_per_call": us,
                    "mean_iterations_run": float(iters.mean()),
                    "us_per_iteration_run": us / max(1.0, iters.max()),
                    "merit_before_mean": float(m[:, 0].mean()),
                    "merit_after_mean": float(m[:, -1].mean()),
                    "merit_reduction_per_us": float((m[:, 0] - m[:, -1]).sum()) / us,
                    "sequences_unsafe_before": int((m[:, 0] > 0).sum()),
                    "sequences_safe_after": int((m[:, -1] == 0).sum()),
                    "device_status_bits": _status_names(bits)}
    return out


def run_curv(args):
    """The curvilinear state variant (s, e_y, e_psi) against the Cartesian model:
    one MPPI iteration (rollouts + update) at K = 65536 and T in {50, 100, 200}
    on the same ellipse track, both from the centreline start; then the shield
    on the curvilinear state: 8192 near-edge sequences, T = 100, 20 iterations
    of the gradient repair (one block per sequence) and of BFGS (one warp per
    sequence), and the full-tape merit gradient."""
    import torch

    import __graft_entry__
    from paper_2302_11719_gb300 import inputs as I
    from paper_2302_11719_gb300 import smppi as S
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rows = []
    K = 65536
    for T in (50, 100, 200):
        for kind, flops in ((0, F_ALG), (1, F_ALG_CURV)):
            pr = I.throughput_problem(K, T)
            if kind == 1:
                pr.params["state_kind"] = 1
                pr.x0 = pr.x0.copy()
                pr.x0[3:6] = 0.0          # s = 0, e_y = 0, e_psi = 0: the same start
            ctl = S.Controller(pr.params, pr.track, device=dev)
            x0, V0 = ctl.tensor(pr.x0), ctl.tensor(pr.V)
            Vb = [V0.clone() for _ in range(args.warmup + 2 * args.steps)]
            for i in range(args.warmup):
                S.smppi_step(ctl.h, x0, Vb[i], i, 0)
            t = _timed_steps(lambda i: S.smppi_step(ctl.h, x0, Vb[args.warmup + i], i, 0),
                             args.steps, flush)
            S.smppi_timing(ctl.h, True)
            _timed_steps(lambda i: S.smppi_step(ctl.h, x0, Vb[args.warmup + args.steps + i], i, 0),
                         args.steps, flush)
            S.smppi_timing(ctl.h, False)
            kt = S.smppi_timing_read(ctl.h)
            st, bits = ctl.sync_status()
            roll_s = kt["rollout"][0] / kt["rollout"][1] / 1e3
            step_s = sum(t) / len(t) / 1e3
            ach = flops * K * T / roll_s / 1e12
            rows.append({"model": "curvilinear" if kind else "cartesian", "K": K, "T": T,
                         "us_per_update": step_s * 1e6, "rollout_steps_per_s": K * T / step_s,
                         "rollout_kernel_us": roll_s * 1e6, "flops_per_rollout_step": flops,
                         "fp32_tflops": ach, "fp32_frac": ach / FP32_PEAK_TFLOPS,
                         "device_status_bits": _status_names(bits)})
            ctl.close()
    sb = I.near_edge_curvilinear(8192, 100, seed=0)
    n = sb.x0.shape[0]
    ctl = S.Controller(sb.params, sb.track, max_seq=n, device=dev)
    x0, V = ctl.tensor(sb.x0), ctl.tensor(sb.V)
    shield = _time_repairs(S, ctl, n, x0, V, 20, args, flush)
    J = torch.empty(n, dtype=torch.float64, device=dev)
    g = torch.empty_like(V)
    for _ in range(args.warmup):
        S.smppi_cost_grad(ctl.h, n, x0, V, 100, 0.0, 1.0, -1, J, g)
    t = _timed_steps(lambda i: S.smppi_cost_grad(ctl.h, n, x0, V, 100, 0.0, 1.0, -1, J, g),
                     args.steps, flush)
    shield["merit_grad_full_tape"] = {"us_per_call": 1e3 * sum(t) / len(t),
                                      "sequence_steps_per_s": n * 100 / (sum(t) / len(t) / 1e3)}
    ctl.close()
    print(json.dumps({"workload": "curvilinear vs Cartesian state, MPPI iteration, K = 65536",
                      "peak_tflops": FP32_PEAK_TFLOPS, "l2": "flushed between steps",
                      "rows": rows,
                      "shield_8192_near_edge_T100": shield}), flush=True)
    return 0


def run_small(args):
    """The small configurations, GPU and FP64 oracle side by side: the K = 256,
    T = 50 Shield-MPPI update (10 Armijo iterations; also the MPPI iteration
    alone) and the K = 1024, T = 60 plain MPPI closed-loop step (no shield, no
    CBF cost)."""
    import torch

    import __graft_entry__
    from paper_2302_11719_gb300 import inputs as I
    from paper_2302_11719_gb300 import smppi as S
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    for name, pr, n_rep in (("shield_update_K256_T50", I.single_step_small(), N_REPAIR),
                            ("plain_step_K1024_T60", I.closed_loop_plain(), 0)):
        ctl = S.Controller(pr.params, pr.track, device=dev)
        x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
        Vs = torch.empty_like(V)
        it = [0]

        def upd(i):
            S.smppi_shield_update(ctl.h, x0, V, Vs, it[0], 0, n_rep)
            it[0] += 1
        for i in range(args.warmup):
            upd(i)
        t = _timed_steps(upd, args.steps, flush)
        row = {"gpu_us_per_update": statistics.median(t) * 1e3}
        if n_rep > 0:
            Vb = [ctl.tensor(pr.V) for _ in range(args.steps)]
            t2 = _timed_steps(lambda i: S.smppi_step(ctl.h, x0, Vb[i], i, 0), args.steps, flush)
            row["gpu_us_mppi_iteration_only"] = statistics.median(t2) * 1e3
        st, bits = ctl.sync_status()
        row["device_status_bits"] = _status_names(bits)
        ctl.close()
        for nt, key in ((cpu_threads(), "oracle_us_per_update_all_cores"),
                        (1, "oracle_us_per_update_1_core")):
            times = oracle_problem_updates(pr, n_rep, 5, nt)
            row[key] = statistics.median(times) * 1e6
        row["cores"] = cpu_threads()
        out[name] = row
    print(json.dumps({"workload": "small configurations (median of the timed steps, L2 flushed "
                                  "between steps; oracle: 5 closed-loop updates on the host)",
                      "results": out}), flush=True)
    return 0


COMPARE_K = (16, 32, 64, 128, 256, 1024)      # rollouts (the paper's samples M)
COMPARE_T = (10, 20, 40, 75)                   # horizon steps of 0.02 s (0.2 .. 1.5 s)
COMPARE_CHUNK = 25                             # updates per graph replay chunk
# narrow tracks (half-width 1-1.5 m), target speed 10 m/s, centring weight 50 and
# disturbances of std 0.2 on (v_y, r): crash rates then span the grid from most
# problems (few rollouts, short horizons) to none (long horizons)
COMPARE_SETTING = dict(w=(1.0, 1.5), v_target=10.0, q_d=50.0, dist_sigma=(0.2, 0.2))


def compare_controllers(S, I, dev, K, T, n_updates, B=128, seed=7, setting=None):
    """One (K, T) cell of the closed-loop comparison: plain MPPI (no DCBF cost,
    no shield), MPPI with the DCBF cost of Eq. 17-20, and Shield-MPPI (DCBF
    cost + up to 10 Armijo repair iterations, Alg. 1), each on the same B
    narrow-track problems from the same starts with the same disturbances
    (Eq. 26), n_updates closed-loop updates in graph replays of COMPARE_CHUNK.
    Returns one row per controller; the device status is checked after every
    chunk."""
    import numpy as np
    import torch
    ctrls = (("plain MPPI", 0.0, 0), ("MPPI + DCBF cost", 1000.0, 0),
             ("Shield-MPPI", 1000.0, N_REPAIR))
    rows = []
    for name, c_cbf, n_rep in ctrls:
        st_ = dict(COMPARE_SETTING if setting is None else setting)
        w_lo, w_hi = st_.pop("w")
        ib = I.uneven_instances(n_inst=B, seed=seed, K_lo=K, K_hi=K, T_lo=T, T_hi=T,
                                w_lo=w_lo, w_hi=w_hi, C_cbf=c_cbf, **st_)
        bt = S.Batch(ib, block_rollouts=0, device=dev)
        S.smppi_batch_loop(bt.b, bt.x0, bt.V, bt.V_safe, 0, n_rep, 1)   # autotune
        S.smppi_batch_sync_status(bt.b)
        bt.x0.copy_(torch.as_tensor(ib.x0, device=dev))
        bt.V.zero_()
        S.smppi_batch_monitor(bt.b, B, reset=True)
        viol = np.zeros(B, np.int64)
        out = np.zeros(B, np.int64)
        ms, bits_seen, done = 0.0, 0, 0
        while done < n_updates:
            n = min(COMPARE_CHUNK, n_updates - done)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record()
            S.smppi_batch_loop(bt.b, bt.x0, bt.V, bt.V_safe, done, n_rep, n)
            a1.record()
            torch.cuda.synchronize()
            ms += a0.elapsed_time(a1)
            st, bits = S.smppi_batch_sync_status(bt.b)
            bits_seen |= bits
            if bits & 2:
                raise RuntimeError("device wait timed out in the %s loop (K=%d, T=%d) after "
                                   "%d updates" % (name, K, T, done + n))
            v, o = S.smppi_batch_monitor(bt.b, B, reset=True)
            viol += v
            out += o
            done += n
        rows.append({"K": K, "T": T, "controller": name,
                     "violation_rate": float(viol.sum()) / (B * n_updates),
                     "outside_rate": float(out.sum()) / (B * n_updates),
                     "crash_rate": float((out > 0).mean()),
                     "ms_per_update_all": ms / n_updates,
                     "status": _status_names(bits_seen)})
        bt.close()
    return rows


def run_compare(args):
    """Closed-loop controller comparison on synthetic tracks (the analogue of the
    paper's Sec. VI-E, whose heat maps cover samples and horizon; the AutoRally
    simulator is not available): plain MPPI, MPPI with the DCBF cost and
    Shield-MPPI on the same 128 narrow-track problems for a grid of rollouts K
    and horizons T.  Rates come from the batch's safety monitor: executed steps
    that break the DCBF condition or end outside the track, and the fraction
    of problems that ever leave the track (a crash)."""
    import torch

    import __graft_entry__
    from paper_2302_11719_gb300 import inputs as I
    from paper_2302_11719_gb300 import smppi as S
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    B, steps = 128, args.loop_updates or 300
    rows = []
    Ks = COMPARE_K if not args.compare_k else tuple(args.compare_k)
    Ts = COMPARE_T if not args.compare_t else tuple(args.compare_t)
    setting = dict(COMPARE_SETTING)
    if args.compare_setting:
        setting.update(json.loads(args.compare_setting))
    for K in Ks:
        for T in Ts:
            rows.extend(compare_controllers(S, I, dev, K, T, steps, B, setting=setting))
    print(json.dumps({"workload": "closed-loop controller comparison, %d problems x %d updates"
                                  % (B, steps),
                      "setting": setting, "rows": rows}), flush=True)
    return 0


def run_grad(args):
    """8192 near-boundary sequences, T = 100: adjoint gradient (checkpoint every
    10 steps vs full tape) and 20 Armijo repair iterations."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2302_11719_gb300 import inputs as I
    from paper_2302_11719_gb300 import smppi as S
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sb = I.near_boundary_sequences(8192, 100, seed=0)
    n = sb.x0.shape[0]
    ctl = S.Controller(sb.params, sb.track, max_seq=n, checkpoint=10, device=dev)
    x0, V = ctl.tensor(sb.x0), ctl.tensor(sb.V)
    J = torch.empty(n, dtype=torch.float64, device=dev)
    g = torch.empty_like(V)
    out = {}
    for name, ck in (("checkpoint_10", 10), ("full_tape", -1)):
        for _ in range(args.warmup):
            S.smppi_cost_grad(ctl.h, n, x0, V, 100, 0.0, 1.0, ck, J, g)
        t = _timed_steps(lambda i: S.smppi_cost_grad(ctl.h, n, x0, V, 100, 0.0, 1.0, ck, J, g),
                         args.steps, flush)
        out[name] = {"us_per_call": 1e3 * sum(t) / len(t),
                     "sequence_steps_per_s": n * 100 / (sum(t) / len(t) / 1e3)}
    # 20 repair iterations: projected gradient + Armijo (mode 1, one thread per
    # sequence at this size) and BFGS (mode 2, one warp per sequence)
    out.update(_time_repairs(S, ctl, n, x0, V, 20, args, flush))
    ctl.close()
    # the FP64 oracle's repairs on a sample of the same sequences (one host core
    # per sequence; sequences are independent, so the whole batch on all cores
    # is extrapolated as sample time x 8192 / 64 / cores)
    import oracle as O
    O.build()
    m = O.Model(sb.params, sb.track)
    n_smp, cores = 64, cpu_threads()
    for key, mode in (("repair_20", 1), ("bfgs_20", 2)):
        a = time.perf_counter()
        for q in range(n_smp):
            O.repair(m, sb.x0[q], sb.V[q], 20, mode=mode)
        dt = time.perf_counter() - a
        out[key]["oracle_fp64_host"] = {
            "sample": "first %d of the %d sequences, one core" % (n_smp, n),
            "us_per_sequence": 1e6 * dt / n_smp,
            "us_per_call_extrapolated_all_cores": 1e6 * dt / n_smp * n / cores,
            "cores": cores}
    # a plain MPPI iteration of the same size (K = 8192 rollouts, T = 100)
    pr = I.throughput_problem(8192, 100)
    c2 = S.Controller(pr.params, pr.track, device=dev)
    x0p, Vp = c2.tensor(pr.x0), c2.tensor(pr.V)
    t = _timed_steps(lambda i: S.smppi_step(c2.h, x0p, Vp.clone(), i, 0), args.steps, flush)
    out["plain_mppi_step_K8192_T100_us"] = 1e3 * sum(t) / len(t)
    c2.close()
    print(json.dumps({"workload": "adjoint gradient and repair, 8192 sequences, T=100",
                      "results": out, "l2": "flushed between calls"}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shield",
                    choices=["shield", "batch", "sweep", "grad", "small", "compare", "curv"])
    ap.add_argument("--loop-updates", type=int, default=None,
                    help="closed-loop updates per problem (batch workload: 500, compare: 300)")
    ap.add_argument("--compare-k", type=int, nargs="*", help="rollouts of the comparison grid")
    ap.add_argument("--compare-t", type=int, nargs="*", help="horizons of the comparison grid")
    ap.add_argument("--shard-rollouts", action="store_true",
                    help="split the K rollouts of one problem over the ranks (strong scaling; "
                         "default: one independent replica per rank)")
    ap.add_argument("--compare-setting", default=None,
                    help="JSON overrides of the comparison's track and cost setting")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--min-timed-seconds", type=float, default=1.2,
                    help="each timed step repeats the update so that the timed region lasts "
                         "at least this long (clock samples under load)")
    ap.add_argument("--active-updates", type=int, default=100,
                    help="updates of the near-boundary (shield-active) workload")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "grad":
        return run_grad(args)
    if args.workload == "small":
        return run_small(args)
    if args.workload == "compare":
        return run_compare(args)
    if args.workload == "curv":
        return run_curv(args)
    if args.shard_rollouts:
        return run_sharded(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
