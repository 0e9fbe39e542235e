#!/usr/bin/env python3
"""Benchmark: value iteration on the large vehicular-cloud placement MDP.

One step = one solve of the resident instance from V = 0 to a certified 1e-6 residual
(Algorithm 3): FP32 Jacobi Bellman sweeps with fused residual, argmax policy, FP64
policy-evaluation refinement and the FP64 Bellman residual check.  The headline form is
the explicit CSR with FP32 probabilities (the HBM-streaming sweep); the implicit
register-generated form is timed beside it.

value  = state-action-successor updates per second = logical nnz per sweep x FP32 sweeps
         / step time (device events on the launching stream, L2 flushed between steps).
e2e    = the same through the public API from host parameters to host results (build,
         solve, copy of V64 and pi back), wall clock.
roofline: the CSR sweep kernel, algorithmic bytes per launch / average launch time.

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "state-action-successor updates/s and time to 1e-6 residual; % of HBM roofline"
UNIT = "updates/s"
WORKLOAD_DESC = {
    "large": "large single MDP: H=7 C=4 Q=15, S=2,500,000 states, A=8 actions, gamma=0.95",
    "tiny": "tiny MDP: H=3 C=3 Q=4, S=640, A=4, gamma=0.95",
    "precision": "precision MDP: H=8 C=4 Q=15, S=12,500,000, A=9, gamma=0.95",
    "grad": "differentiation MDP: H=6 C=4 Q=10, S=343,750, A=7, gamma=0.95",
    "medium": "medium MDP: H=7 C=3 Q=15, S=524,288, A=8, gamma=0.95 (the large MDP's structure at a fifth of "
              "its size: stored matrix above L2, under 1 GB on the device)",
    "batched": "512 uneven instances: H in 2..5, C in 2..6, Q in 3..12, gamma in {0.9, 0.95, 0.99}, "
               "S in [72, 436,982]",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOAD_DESC))
    ap.add_argument("--form", default="csr_f32", choices=["csr_f32", "csr_bf16", "implicit"])
    ap.add_argument("--layout", default="padded", choices=["padded", "canonical"],
                    help="padded: every row holds 2H+3 entries (340,000,000 per sweep on the large MDP, the "
                         "workload's stated CSR size); canonical: only non-zero successors (130,468,750)")
    ap.add_argument("--no-sliced", dest="sliced", action="store_false",
                    help="CSR kernels only: build no sliced (SELL-C-sigma) copy of the stored matrix for the "
                         "autotuner to choose")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--self-loop", dest="self_loop", action="store_true",
                    help="FP32 sweeps solve each action's self-transition exactly (VC_ITER_SELF_LOOP; same V*, "
                         "fewer sweeps); by default the step runs Eq. 18's backup as Algorithm 3 states it")
    ap.add_argument("--block", action="store_true",
                    help="implicit form only: FP32 sweeps run Algorithm 4's in-block iteration (VC_ITER_BLOCK, the "
                         "handle's default block shape)")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, cpu baseline and the variants")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default CSR schedule (profiling runs: no tuning launches before the timed ones)")
    args = ap.parse_args()
    args.padded = args.layout == "padded" and args.form != "implicit"
    args.sliced = args.sliced and args.form != "implicit"
    if args.block and args.form != "implicit":
        ap.error("--block needs --form implicit")
    return args


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- native arm
def run_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2012_12419_gb300 import inputs, native

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    native.load(build_if_missing=(rank == 0))
    if world > 1:
        dist.barrier()
        native.load()

    p = inputs.workload(args.workload)
    t0 = time.perf_counter()
    m = native.MDP.build(p, fmt=args.form, padded=args.padded, sliced=args.sliced)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3
    tune_us = m.autotune(reps=5) if (args.form != "implicit" and not args.no_autotune) else None
    tune_report = m.autotune_report() if tune_us is not None else None
    info = m.info()
    S = int(info["S"])
    nnz = int(info["nnz_logical"])
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    V = torch.zeros(S, dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2

    def step():
        V.zero_()  # Algorithm 3, step 1
        _, V64, pi, st = m.value_iterate(V, tol=args.tol, self_loop=args.self_loop, block=args.block)
        return st

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = native.kernel_launches()
    times, stats = [], []
    region0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step()
        e1.record(stream)
        stats.append(st)
        times.append((e0, e1))
    torch.cuda.synchronize()
    region_s = time.perf_counter() - region0
    launches = native.kernel_launches() - launches0
    ck = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in times]
    total_ms = sum(ms)
    sweeps = [s["sweeps"] for s in stats]
    units = float(nnz) * float(sum(sweeps))
    if world > 1:
        t = torch.tensor([total_ms, units], dtype=torch.float64, device=dev)
        tmax = t.clone()
        dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        total_ms_all, units_all = float(tmax[0]), float(t[1])
        dist.barrier()
    else:
        total_ms_all, units_all = total_ms, units
    value = units_all / (total_ms_all / 1e3)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": step_config(args, nnz, world),
        "layout": layout_of(args, info),
        "time_to_residual_ms": statistics.median(ms),
        "sweeps_per_step": statistics.median(sweeps),
        "fp32_correction_products_per_step": statistics.median([s["eval_sweeps"] for s in stats]),
        "fp64_backups_per_step": statistics.median([s["bellman64"] for s in stats]),
        "policy_rounds_per_step": statistics.median([s["policy_rounds"] for s in stats]),
        "ms_fp32_sweeps": statistics.median([s["ms_fp32"] for s in stats]),
        "ms_fp64_refine": statistics.median([s["ms_fp64"] for s in stats]),
        "certified": all(s["certified"] == 1 for s in stats),
        "residual64": max(s["residual64"] for s in stats),
        "build_ms": build_ms,
        "autotuned_sweep_us": tune_us,
        "autotune": tune_report.strip().splitlines() if tune_report else None,
        "gpu_launches": int(launches),
        "region_wall_s": region_s,
        "clocks": ck,
    }
    if rank == 0:
        out["roofline"] = roofline(m, info, args, V, dev, stream)
        if not args.no_extras:
            out["e2e"] = e2e(args, p, native, torch, nnz)
            if world == 1:
                out["cpu_baseline"] = cpu_baseline(p, args)
            out["variants"] = variants(args, p, native, torch, dev, stream)
            out["self_loop"] = self_loop_comparison(args, p, m, V, native, torch, dev, stream)
            if world == 1 and args.workload == "large":
                out["comparisons"] = comparisons(args, native, torch, dev, stream)
                out["batched"] = batched_record(args, native, torch, dev, stream)
                out["binary_model"] = binary_record(args, native, torch, dev, stream)
        print(json.dumps(out))
    m.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def step_config(args, nnz_logical, world):
    """The workload and step definition, identical in both arms (the reference arm times the
    oracle on the same workload, so nothing here names an implementation's storage)."""
    return {
        "workload": WORKLOAD_DESC[args.workload],
        "form": args.form + ("+padded" if args.padded else "") + ("+sliced" if args.sliced else ""),
        "tol": args.tol, "nnz_logical_per_sweep": int(nnz_logical),
        "parallelism": "replicas" if world > 1 else "single",
        "l2": "256 MiB buffer written between steps, outside the step events",
        "step": "V=0 -> FP32 sweeps -> argmax -> FP64 policy evaluation -> FP64 Bellman certificate",
        "sweep": ("in-block iteration, self-transitions solved" if getattr(args, "block", False) else
                  "self-transition solved" if args.self_loop else "Eq. 18 backup"),
    }


def layout_of(args, info):
    """What the timed sweep streams: the stored matrix and, when the sweep runs on it, the
    sliced copy (which drops infeasible rows and pads each 32-state block to its longest row)."""
    sliced = bool(info["csr_sliced"])
    nnz_stored = int(info["nnz_stored"])
    d = {"nnz_stored_matrix": nnz_stored, "nnz_streamed_per_sweep": int(info["nnz_sliced"]) if sliced else nnz_stored,
         "stored_bytes_per_sweep": int(info["sweep_bytes"])}
    if args.form == "implicit":
        d["streamed"] = "nothing per transition: successors generated in registers from the state code"
    elif sliced:
        d["streamed"] = (f"sliced copy of the {'padded' if args.padded else 'canonical'} CSR ({nnz_stored:,} "
                         f"entries): infeasible rows and explicit zeros dropped, each 32-state block padded to its "
                         f"longest row, {int(info['nnz_sliced']):,} entries")
    else:
        d["streamed"] = f"{'padded' if args.padded else 'canonical'} CSR, {nnz_stored:,} entries"
    return d


def algorithmic_sweep_bytes(S, A, nnz_logical, bf16):
    """Algorithmic HBM bytes of one explicit Bellman sweep of the logical (canonical) work:
    each non-zero successor's value and column, each (state, action) row's offset and
    reward (and BF16 row scale), V read and written once."""
    v = 2 if bf16 else 4
    return nnz_logical * (v + 4) + S * A * (8 + 4 + (4 if bf16 else 0)) + 8 * S


# --------------------------------------------------------------------------- batched arm
def _implicit_nnz(native, p):
    """Logical successor count per sweep of one instance (canonical, feasible rows)."""
    m = native.MDP.build(p, fmt="implicit")
    n = int(m.info()["nnz_logical"])
    m.close()
    return n


def run_batched(args):
    """512 uneven instances in one graph-captured persistent solve (per-instance gamma and
    termination).  Under torchrun the instances are split across ranks by the LPT rule and
    each rank solves its share; value = all ranks' updates / the slowest rank's time."""
    import torch
    import torch.distributed as dist

    from paper_2012_12419_gb300 import inputs, native, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    native.load(build_if_missing=(rank == 0))
    if world > 1:
        dist.barrier()
        native.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ps_all = inputs.batch_params(512, seed=2)
    idx, ps = shard.shard_of(ps_all, rank, world, args.tol)
    nnz = [_implicit_nnz(native, p) for p in ps]
    t0 = time.perf_counter()
    b = native.Batch(ps)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3
    tune_ms = b.autotune(sweeps=20) if not args.no_autotune else None
    tune_sweep_ms = tune_ms / 20 if tune_ms else None
    binfo = b.info()
    V = torch.zeros(b.total, dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        V.zero_()
        _, _, _, st, _ = b.value_iterate(V, tol=args.tol, self_loop=args.self_loop)
        return st

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = native.kernel_launches()
    times, stats = [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step()
        e1.record(stream)
        stats.append(st)
        times.append((e0, e1))
    torch.cuda.synchronize()
    launches = native.kernel_launches() - launches0
    ck = clocks.stop()
    ms = [a.elapsed_time(c) for a, c in times]
    total_ms = sum(ms)
    units = float(sum(n * s["sweeps"] for st in stats for n, s in zip(nnz, st)))
    if world > 1:
        t = torch.tensor([total_ms, units], dtype=torch.float64, device=dev)
        tmax = t.clone()
        dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        total_ms_all, units_all = float(tmax[0]), float(t[1])
        gathered = shard.gather_by_index({i: (s["sweeps"], s["certified"]) for i, s in zip(idx, stats[-1])},
                                         len(ps_all))
    else:
        total_ms_all, units_all = total_ms, units
        gathered = [(s["sweeps"], s["certified"]) for s in stats[-1]]
    last = stats[-1]
    out = {
        "metric": METRIC, "value": units_all / (total_ms_all / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_ms_all / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": WORKLOAD_DESC["batched"], "form": "implicit, batched graph",
            "tol": args.tol, "instances": len(ps_all), "instances_this_rank": len(ps),
            "states_this_rank": int(binfo["total_states"]),
            "parallelism": f"LPT split over {world} ranks" if world > 1 else "single",
            "l2": "256 MiB buffer written between steps, outside the step events",
            "step": "V=0 -> one graph launch of FP32 sweeps with per-instance termination -> argmax -> "
                    "FP64 policy evaluation -> FP64 Bellman certificate per instance",
            "sweep": "self-transition solved" if args.self_loop else "Eq. 18 backup",
        },
        "time_to_residual_ms": statistics.median(ms),
        "certified": all(c == 1 for _, c in gathered),
        "sweeps_max": max(s for s, _ in gathered), "sweeps_median": statistics.median([s for s, _ in gathered]),
        "residual64": max(s["residual64"] for s in last),
        "build_ms": build_ms,
        "schedule": {k: int(binfo[k]) for k in ("tile_states", "blocks_per_sm", "grid", "tiles")},
        "whole_instance_in_one_block": b.small_instances(),
        "autotune": b.autotune_report().strip().splitlines() if tune_ms else None,
        "gpu_launches": int(launches),
        "clocks": ck,
    }
    if rank == 0 and tune_sweep_ms:
        hbm, src = peaks()
        nbytes = 8 * int(binfo["total_states"])
        ach = nbytes / (tune_sweep_ms / 1e3) / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                           "traffic": None, "peak_source": f"{src} hbm_gbs",
                           "kernel": "k_bpost+k_bmax (one graph pass = one sweep of every instance)",
                           "bytes_per_launch": nbytes, "launch_us": tune_sweep_ms * 1e3,
                           "ncu_sol": batched_sol()}
    if rank == 0 and not args.no_extras:
        out["e2e"] = batched_e2e(args, ps, nnz, native, torch)
        if world == 1:
            out["cpu_baseline"] = cpu_baseline_batched(ps_all)
            out["vs_per_instance"] = batched_vs_per_instance(args, ps, b, native, torch, dev, stream)
            out["self_loop"] = batched_self_loop(args, b, torch, dev, stream)
    if rank == 0:
        print(json.dumps(out))
    b.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def binary_record(args, native, torch, dev, stream):
    """The paper's binary-action model (A = {-1, 1}: paid traditional cloud or the
    requested vehicular cloud; 6 clouds of 6 VMs, requests of 1-3 VMs, 2,235,331 states) as
    an explicit CSR built on the device, solved to the certified residual in each storage
    form, device-timed like the headline step, with the sweep's roofline."""
    from paper_2012_12419_gb300 import inputs

    p = inputs.binary_workload("binary")
    hbm, src = peaks()
    out = {"workload": "binary-action model: H=6 clouds x C=6 VMs, requests of 1..3 VMs, S=2,235,331, A=2, "
                       "gamma=0.95"}
    for form, sliced in (("csr_f32", True), ("csr_f32", False), ("csr_bf16", True)):
        t0 = time.perf_counter()
        m = native.MDP.build_binary(p, fmt=form, sliced=sliced)
        torch.cuda.synchronize()
        build_ms = (time.perf_counter() - t0) * 1e3
        m.autotune(reps=5)
        info = m.info()
        V = torch.zeros(info["S"], dtype=torch.float32, device=dev)
        res = {}
        for sl in (False, True):
            def solve():
                V.zero_()
                return m.value_iterate(V, tol=args.tol, self_loop=sl)

            solve()
            t, (_, _, _, st) = _timed(torch, stream, solve, 3)
            res[sl] = (t, st)
        best = _best_plan(m)
        sweep_us = float(best.split()[-1]) if best else None
        alg = algorithmic_sweep_bytes(int(info["S"]), 2, int(info["nnz_logical"]), form == "csr_bf16")
        t, st = res[False]
        out[form + ("+sliced" if sliced else "")] = {
            "time_to_residual_ms": t, "sweeps": int(st["sweeps"]), "certified": st["certified"] == 1,
            "updates_per_s": info["nnz_logical"] * st["sweeps"] / (t / 1e3),
            "ms_fp32_sweeps": st["ms_fp32"], "ms_fp64_refine": st["ms_fp64"], "build_ms": build_ms,
            "sweep_us": sweep_us, "alg_bytes_per_sweep": alg,
            "sweep_frac": (alg / (sweep_us * 1e-6) / 1e9 / hbm) if sweep_us else None,
            "stored_frac": (info["sweep_bytes"] / (sweep_us * 1e-6) / 1e9 / hbm) if sweep_us else None,
            "peak_source": f"{src} hbm_gbs",
            "self_loop_ms": res[True][0], "self_loop_sweeps": int(res[True][1]["sweeps"]),
            "self_loop_certified": res[True][1]["certified"] == 1,
            "nnz_logical": int(info["nnz_logical"]), "nnz_sliced": int(info["nnz_sliced"]), "tuned": best}
        m.close()
    return out


def batched_record(args, native, torch, dev, stream, steps: int = 5):
    """The 512-instance batched workload inside the default run: one graph-captured solve of
    every instance to its certified residual, timed as the batched arm times it (L2 flushed
    between steps, events on the stream), with the per-instance plain-FP32 comparison and
    the self-transition variant."""
    from paper_2012_12419_gb300 import inputs

    ps = inputs.batch_params(512, seed=2)
    nnz = [_implicit_nnz(native, p) for p in ps]
    b = native.Batch(ps)
    tune_ms = b.autotune(sweeps=20)
    binfo = b.info()
    V = torch.zeros(b.total, dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        V.zero_()
        return b.value_iterate(V, tol=args.tol)[3]

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ms, stats = [], []
    for k in range(steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    units = float(sum(n * x["sweeps"] for st in stats for n, x in zip(nnz, st)))
    last = stats[-1]
    out = {
        "workload": WORKLOAD_DESC["batched"], "value": units / (sum(ms) / 1e3), "unit": UNIT, "steps": steps,
        "ms_per_step": sum(ms) / steps, "time_to_residual_ms": statistics.median(ms),
        "states": int(binfo["total_states"]), "certified": all(x["certified"] == 1 for x in last),
        "sweeps_max": max(x["sweeps"] for x in last), "sweeps_median": statistics.median([x["sweeps"] for x in last]),
        "residual64": max(x["residual64"] for x in last),
        "schedule": {k: int(binfo[k]) for k in ("tile_states", "blocks_per_sm", "grid", "tiles")},
        "autotuned_sweep_ms": tune_ms / 20,
        "whole_instance_in_one_block": b.small_instances(),
    }
    out["vs_per_instance"] = batched_vs_per_instance(args, ps, b, native, torch, dev, stream)
    out["self_loop"] = batched_self_loop(args, b, torch, dev, stream)
    b.close()
    return out


def batched_self_loop(args, b, torch, dev, stream):
    """The batched step with and without VC_ITER_SELF_LOOP (each instance's FP32 loop solves
    every action's self-transition exactly), device-timed to the same certified residual."""
    V = torch.zeros(b.total, dtype=torch.float32, device=dev)
    res = {}
    for sl in (False, True):
        def solve():
            V.zero_()
            return b.value_iterate(V, tol=args.tol, self_loop=sl)

        solve()
        t, (_, V64, _, st, _) = _timed(torch, stream, solve, 3)
        res[sl] = (t, V64.clone(), st)
    (t0, V0, s0), (t1, V1, s1) = res[False], res[True]
    out = {"eq18_ms": t0, "self_loop_ms": t1, "speedup": t0 / t1,
           "eq18_sweeps_total": int(sum(x["sweeps"] for x in s0)),
           "self_loop_sweeps_total": int(sum(x["sweeps"] for x in s1)),
           "certified": all(x["certified"] == 1 for x in s0 + s1),
           "max_abs_V64_difference": float((V1 - V0).abs().max())}
    # Algorithm 4's in-block passes on every instance (blocks of at most `threads` states)
    shapes, best = [], None
    for threads, passes in ((256, 2), (256, 4), (512, 2), (512, 4), (512, 8)):
        b.set_block_iteration(threads, passes)

        def solve():
            V.zero_()
            return b.value_iterate(V, tol=args.tol, block=True)

        solve()
        t, (_, _, _, st, _) = _timed(torch, stream, solve, 3)
        row = {"threads": threads, "passes": passes, "ms": t, "sweeps_total": int(sum(x["sweeps"] for x in st)),
               "sweeps_max": int(max(x["sweeps"] for x in st)), "certified": all(x["certified"] == 1 for x in st)}
        shapes.append(row)
        if best is None or t < best["ms"]:
            best = row
    b.set_block_iteration(512, 4)
    out["block"] = {"shapes": shapes, "best": best, "speedup_vs_self_loop": t1 / best["ms"],
                    "speedup_vs_eq18": t0 / best["ms"]}
    return out


def batched_e2e(args, ps, nnz, native, torch):
    """Public API from host parameters to host results, every step: batch build (H2D of the
    parameter structs and rate arrays), solve, D2H of V64 and pi into pinned buffers."""
    import ctypes

    from paper_2012_12419_gb300 import inputs

    T = sum(inputs.num_states(p["H"], p["C"], p["Q"]) for p in ps)
    hv = torch.empty(T, dtype=torch.float64, pin_memory=True)
    hp = torch.empty(T, dtype=torch.int32, pin_memory=True)
    ms, units = [], []
    for _ in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = native.Batch(ps)
        _, V64, pi, st, _ = b.value_iterate(tol=args.tol, self_loop=args.self_loop)
        hv.copy_(V64, non_blocking=True)
        hp.copy_(pi, non_blocking=True)
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
        units.append(sum(n * x["sweeps"] for n, x in zip(nnz, st)))
        b.close()
    ms, units = ms[1:], units[1:]  # the first call warms the allocator
    h2d = sum(ctypes.sizeof(native.Params) + 16 * int(p["H"]) for p in ps)
    return {"value": sum(units) / (sum(ms) / 1e3), "unit": UNIT, "ms_per_step": statistics.median(ms),
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(hv.numel()) * 12}


def _timed(torch, stream, fn, reps):
    """Median device time (events on the launching stream) of fn() over reps calls."""
    ms, last = [], None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        last = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms), last


def batched_vs_per_instance(args, ps, b, native, torch, dev, stream):
    """The batched graph solve against the plain FP32 form: every instance solved on its
    own (implicit FP32 sweeps, same certification), one after another on the same GPU."""
    ms_b, (_, V64b, _, stb, _) = _timed(torch, stream, lambda: b.value_iterate(tol=args.tol), 3)
    ms_ba, (_, V64a, _, sta, _) = _timed(torch, stream, lambda: b.value_iterate(tol=args.tol, accurate=True), 3)
    ms_ff, _ = _timed(torch, stream, lambda: b.value_iterate(tol=args.tol, fp32_only=True), 3)
    ms_ = [native.MDP.build(p, fmt="implicit") for p in ps]
    for m in ms_:
        m.value_iterate(tol=args.tol)

    def solo():
        return [m.value_iterate(tol=args.tol) for m in ms_]

    ms_s, res = _timed(torch, stream, solo, 2)
    off = b.offsets
    dv = 0.0
    for i, (_, V64s, _, st) in enumerate(res):
        dv = max(dv, float((V64b[off[i]:off[i + 1]] - V64s).abs().max()))
    for m in ms_:
        m.close()
    return {
        "per_instance_fp32_ms": ms_s, "batched_ms": ms_b, "speedup": ms_s / ms_b,
        "batched_fp32_loop_only_ms": ms_ff, "batched_accurate_ms": ms_ba,
        "per_instance_sweeps_total": int(sum(r[3]["sweeps"] for r in res)),
        "batched_sweeps_total": int(sum(s["sweeps"] for s in stb)),
        "max_abs_V64_batched_minus_per_instance": dv,
        "all_certified": all(s["certified"] == 1 for s in stb) and all(r[3]["certified"] == 1 for r in res),
        "accurate_all_certified": all(s["certified"] == 1 for s in sta),
        "note": "per-instance = vc_value_iterate on each of the instances in turn (implicit FP32 form)",
    }


def cpu_baseline_batched(ps_all, min_seconds: float = 6.0):
    """The FP64 oracle's Bellman sweeps over the batch's instances (one sweep of each, in
    order), single thread and with the instances spread over every host core."""
    import threading

    import numpy as np

    import oracle

    cores = os.cpu_count() or 1

    def one(p):
        S = oracle.num_states(p)
        return oracle.sweep_states(p, np.zeros(S), np.zeros(S), 0, S, 1)

    u1, n1 = 0, 0
    t0 = time.perf_counter()
    for p in ps_all:
        u1 += one(p)
        n1 += 1
        if time.perf_counter() - t0 > min_seconds:
            break
    t1 = time.perf_counter() - t0
    counts = [0] * cores

    def work(k):
        counts[k] = sum(one(p) for p in ps_all[k::cores])

    t0 = time.perf_counter()
    ts = [threading.Thread(target=work, args=(k,)) for k in range(cores)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    tn = time.perf_counter() - t0
    un = sum(counts)
    return {"value": un / tn, "unit": UNIT, "cores": cores, "kind": "oracle", "single_thread_value": u1 / t1,
            "sample": f"one Jacobi sweep from V=0 of each of the {len(ps_all)} instances on {cores} threads "
                      f"({un} updates, {tn:.1f} s); single thread: the first {n1} instances ({u1} updates, "
                      f"{t1:.1f} s)"}


def comparisons(args, native, torch, dev, stream):
    """BF16 storage and the adjoint gradient, each timed against the plain FP32 form on the
    same GPU at the same certified residual."""
    from paper_2012_12419_gb300 import inputs

    out = {}
    p = inputs.workload("precision")
    res = {}
    for layout in ("padded", "canonical", "padded+sliced", "canonical+sliced"):
        for form in ("csr_f32", "csr_bf16"):
            m = native.MDP.build(p, fmt=form, padded=layout.startswith("padded"), sliced=layout.endswith("sliced"))
            m.autotune(reps=3)
            info = m.info()
            V = torch.zeros(info["S"], dtype=torch.float32, device=dev)

            def solve():
                V.zero_()
                return m.value_iterate(V, tol=args.tol)

            solve()
            t, (_, V64, _, st) = _timed(torch, stream, solve, 2)
            res[(layout, form)] = V64
            out[f"precision_{form}_{layout}"] = {
                "time_to_residual_ms": t, "sweeps": int(st["sweeps"]), "ms_fp32_sweeps": st["ms_fp32"],
                "ms_fp64_refine": st["ms_fp64"], "certified": st["certified"] == 1,
                "updates_per_s": info["nnz_logical"] * st["sweeps"] / (t / 1e3),
                "sweep_bytes": int(info["sweep_bytes"]), "nnz_stored": int(info["nnz_stored"])}
            m.close()
        f32, bf = res[(layout, "csr_f32")], res[(layout, "csr_bf16")]
        out[f"precision_{layout}_bf16_speedup"] = (out[f"precision_csr_f32_{layout}"]["time_to_residual_ms"]
                                                   / out[f"precision_csr_bf16_{layout}"]["time_to_residual_ms"])
        out[f"precision_{layout}_bf16_minus_f32_max_rel"] = float(((bf - f32).abs() / f32.abs().clamp_min(1.0)).max())
    res.clear()

    g = inputs.workload("grad")
    m = native.MDP.build(g, fmt="implicit")
    S = m.S
    rho = torch.zeros(S, dtype=torch.float64, device=dev)
    rho[: 2 * (g["Q"] + 1)] = 1.0 / (2 * (g["Q"] + 1))  # uniform over the states with every host empty
    t_fwd, (_, V64, pi, st) = _timed(torch, stream, lambda: m.value_iterate(tol=args.tol), 3)
    t_adj, (dJ, _, gs) = _timed(torch, stream, lambda: m.value_grad(V64, pi, rho, tol=args.tol), 3)
    t_adj11, (dJ11, _, gs11) = _timed(torch, stream, lambda: m.value_grad(V64, pi, rho, tol=1e-11), 3)
    out["grad_forward_fp32_ms"] = t_fwd
    out["grad_adjoint_ms"] = t_adj
    out["grad_adjoint_over_forward"] = t_adj / t_fwd
    out["grad_adjoint_tol1e-11_ms"] = t_adj11
    out["grad_adjoint_products"] = int(gs["sweeps"]) + int(gs["correction_sweeps"])
    out["grad_forward_sweeps"] = int(st["sweeps"])
    out["grad_nnz_transpose"] = int(gs["nnz_transpose"])
    out["grad_max_abs_dJ_tol1e-6_minus_tol1e-11"] = float((dJ - dJ11).abs().max())
    m.close()

    # the paper's comparison: the greedy heuristic (Algorithm 2 as a policy) against the
    # optimum, on the large workload, J = uniform over the states with every host empty
    p = inputs.workload("large")
    m = native.MDP.build(p, fmt="implicit")
    _, V64, _, st = m.value_iterate(tol=args.tol)
    t_g, pig = _timed(torch, stream, lambda: m.greedy_policy(), 3)
    t_e, (Vg, n_e) = _timed(torch, stream, lambda: m.evaluate_policy(pig, tol=args.tol), 2)
    rho = torch.zeros(m.S, dtype=torch.float64, device=dev)
    rho[: 2 * (p["Q"] + 1)] = 1.0 / (2 * (p["Q"] + 1))
    out["greedy_J"] = float(rho @ Vg)
    out["optimal_J"] = float(rho @ V64)
    out["greedy_policy_ms"] = t_g
    out["greedy_eval_ms"] = t_e
    out["greedy_eval_sweeps"] = int(n_e)
    out["greedy_never_above_optimum"] = bool(torch.all(Vg <= V64 + 2 * p["gamma"] / (1 - p["gamma"]) * args.tol))
    m.close()
    return out


# DRAM bytes (read + write) per launch of the headline sweep kernels, from one ncu capture
# of this exact kernel source each (large workload, padded and canonical CSR with the sliced
# copy); reported only while the sources hash the same, since a changed kernel voids them.
TRAFFIC_SOURCES = ("vc_sell.cu", "vc_internal.cuh", "vc_ptx.cuh")
TRAFFIC_SOURCE_SHA = "ccd123720a0440f4264ecffae2b2e4c7708db65c275981d09ba7e4ea54b0bf9c"
TRAFFIC_BYTES = {("large", "csr_f32", True, True): 1_196_185_088,
                 ("large", "csr_f32", False, True): 1_195_722_752}


# ncu speed-of-light figures of the batched loop's pass-1 kernel on the 512-instance batch,
# attached to the batched roofline while the sources hash as captured: that sweep is bound
# by gather latency at half occupancy, not by a memory roof, and these say how far each
# unit is from its own peak.
BATCH_SOL_SOURCES = ("vc_batch.cu", "vc_internal.cuh")
BATCH_SOL_SHA = "e67621a040703bc539f2e76a5369e75f8b8b8f6eb229700aff8d1bdc6019604b"
BATCH_SOL = {"kernel": "k_bpost_pair<5>", "dram_pct": 11.5, "l2_pct": 13.1, "sm_pct": 57.5,
             "warps_active_pct": 34.6, "registers_per_thread": 80, "top_stall": "long scoreboard (V gathers)"}


def _sources_sha(names):
    import hashlib

    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2012_12419_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic(args, info):
    """(bytes per launch, provenance) of the timed kernel from its ncu capture, or (None, why)."""
    key = (args.workload, args.form, args.padded, bool(info["csr_sliced"]))
    if key not in TRAFFIC_BYTES or not info["csr_pipelined"]:
        return None, "no capture of this configuration"
    sha = _sources_sha(TRAFFIC_SOURCES)
    if sha != TRAFFIC_SOURCE_SHA:
        return None, "kernel sources changed since the capture"
    return TRAFFIC_BYTES[key], f"ncu dram__bytes_read.sum + dram__bytes_write.sum, sources sha256 {sha[:16]}"


# ncu speed-of-light figures of the implicit sweep's two kernels on the large workload,
# attached to that variant while the kernel source hashes as captured: the sweep is bound
# by gather latency and issue, not by a memory roof (its HBM fraction is low by design).
IMPLICIT_SOL_SOURCES = ("vc_sweep.cu",)
IMPLICIT_SOL_SHA = "79e3021f39c95e9a34dc40bbf3e7c264ba4567f09c922b7da7e06a346d0060c7"
IMPLICIT_SOL = {"kernels": "k_post_pair<7, 0> / k_max_pair<7, 0>", "sm_pct": [55.0, 43.0],
                "l2_pct": [14.7, 9.7], "dram_pct": [5.8, 9.1], "warps_active_pct": [49.6, 55.5],
                "top_stall": ["not selected (issue-bound)", "long scoreboard (U gathers)"],
                "bound": "instruction issue (pass 1) and gather latency (pass 2)"}


def implicit_sol():
    return dict(IMPLICIT_SOL) if _sources_sha(IMPLICIT_SOL_SOURCES) == IMPLICIT_SOL_SHA else None


def _sweep_us(m, torch, dev, stream, n: int = 40):
    """Average time of one FP32 sweep (every kernel of it), events on the stream."""
    S = int(m.info()["S"])
    A = torch.rand(S, dtype=torch.float32, device=dev) * 50
    B = torch.empty_like(A)
    for _ in range(5):
        m.bellman32(A, B, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(n):
        if i % 2 == 0:
            m.bellman32(A, B, stream=stream)
        else:
            m.bellman32(B, A, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e3 / n


def batched_sol():
    return dict(BATCH_SOL) if _sources_sha(BATCH_SOL_SOURCES) == BATCH_SOL_SHA else None


def roofline(m, info, args, V, dev, stream):
    """Average launch time of the FP32 sweep kernel, timed with events on its stream.

    frac = algorithmic bytes of the logical work (every non-zero successor once, the
    canonical count) / launch time / measured HBM copy bandwidth; stored_frac = the bytes
    the timed layout actually stores per sweep over the same time."""
    import torch

    hbm, src = peaks()
    A = torch.rand(info["S"], dtype=torch.float32, device=dev) * 50
    B = torch.empty_like(A)
    for _ in range(5):
        m.bellman32(A, B, stream=stream)
    n = 50
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(n):
        if i % 2 == 0:
            m.bellman32(A, B, stream=stream)
        else:
            m.bellman32(B, A, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    avg_s = e0.elapsed_time(e1) / 1e3 / n
    implicit = args.form == "implicit"
    S, Aa = int(info["S"]), int(info["A"])
    if implicit:
        alg = 8 * S  # V read and written; no matrix
    else:
        alg = algorithmic_sweep_bytes(S, Aa, int(info["nnz_logical"]), args.form == "csr_bf16")
    traffic, provenance = captured_traffic(args, info)
    achieved = alg / avg_s / 1e9
    stored = info["sweep_bytes"] / avg_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "traffic_source": provenance, "peak_source": f"{src} hbm_gbs",
            "kernel": "k_post+k_max" if implicit else (
                ("k_sell_ring" if info["csr_pipelined"] else "k_sell") if info["csr_sliced"]
                else ("k_csr_tma" if info["csr_pipelined"] else "k_csr_direct")),
            "bytes_per_launch": int(alg),
            "bytes_definition": "8 S (V in and out)" if implicit else
            "logical nnz x (value + 4 B column) + S A x (8 B offset + 4 B reward [+ 4 B BF16 scale]) + 8 S",
            "launch_us": avg_s * 1e6,
            "stored_bytes_per_launch": int(info["sweep_bytes"]), "stored_achieved": stored,
            "stored_frac": stored / hbm,
            "plan": {k: int(info[k]) for k in ("csr_pipelined", "csr_tile_states", "csr_stages", "csr_ctas_per_sm",
                                                "csr_smem_bytes")}}


def e2e(args, p, native, torch, nnz):
    """Public API from host parameters to host results, every step: build (H2D of the
    parameters; the CSR, its sliced copy and the schedule on the device), solve, D2H of V64
    and pi into pinned buffers allocated once before the steps."""
    from paper_2012_12419_gb300 import inputs

    reps = min(3, args.steps)
    S = inputs.num_states(p["H"], p["C"], p["Q"])
    hv = torch.empty(S, dtype=torch.float64, pin_memory=True)
    hp = torch.empty(S, dtype=torch.int32, pin_memory=True)
    ms, build, sw = [], [], []
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = native.MDP.build(p, fmt=args.form, padded=args.padded, sliced=args.sliced)
        torch.cuda.synchronize()
        tb = time.perf_counter()
        V, V64, pi, st = m.value_iterate(tol=args.tol, self_loop=args.self_loop, block=args.block)
        hv.copy_(V64, non_blocking=True)
        hp.copy_(pi, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        m.close()
        ms.append((t1 - t0) * 1e3)
        build.append((tb - t0) * 1e3)
        sw.append(st["sweeps"])
    ms, build, sw = ms[1:], build[1:], sw[1:]  # first call warms allocator and module
    h2d = 8 * (2 * int(p["H"]) + 8)  # parameter struct and rate arrays
    d2h = S * (8 + 4)
    return {"value": nnz * sum(sw) / (sum(ms) / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": statistics.median(ms),
            "build_ms": statistics.median(build)}


def _best_plan(m):
    """The autotuner's chosen line (kernel, tile, stages, CTAs/SM, smem, us per sweep)."""
    rows = m.autotune_report().strip().splitlines()[1:]
    return min(rows, key=lambda r: float(r.split()[-1])) if rows else None


def self_loop_comparison(args, p, m, V, native, torch, dev, stream):
    """The same step with and without VC_ITER_SELF_LOOP (FP32 sweeps that solve each
    action's self-transition exactly), on the bench's handle and on the implicit form, each
    device-timed to the same certified residual."""
    out = {}
    mi = native.MDP.build(p, fmt="implicit")
    Vi = torch.zeros(int(mi.info()["S"]), dtype=torch.float32, device=dev)
    for name, mm, Vb in (("bench_form", m, V), ("implicit", mi, Vi)):
        res = {}
        for sl in (False, True):
            def solve():
                Vb.zero_()
                return mm.value_iterate(Vb, tol=args.tol, self_loop=sl)

            solve()
            t, (_, V64, _, st) = _timed(torch, stream, solve, 3)
            res[sl] = (t, V64.clone(), st)
        (t0, V0, s0), (t1, V1, s1) = res[False], res[True]
        out[name] = {
            "eq18_ms": t0, "self_loop_ms": t1, "speedup": t0 / t1,
            "eq18_sweeps": int(s0["sweeps"]), "self_loop_sweeps": int(s1["sweeps"]),
            "self_loop_ms_fp32_sweeps": s1["ms_fp32"], "self_loop_ms_fp64_refine": s1["ms_fp64"],
            "self_loop_us_per_sweep": 1e3 * s1["ms_fp32"] / max(int(s1["sweeps"]), 1),
            "eq18_us_per_sweep": 1e3 * s0["ms_fp32"] / max(int(s0["sweeps"]), 1),
            "certified": s0["certified"] == 1 and s1["certified"] == 1,
            "max_abs_V64_difference": float((V1 - V0).abs().max()),
        }
    out["implicit"]["block"] = block_comparison(args, mi, Vi, torch, stream, res[True][0])
    mi.close()
    return out


def block_comparison(args, mi, Vi, torch, stream, t_self_loop):
    """Algorithm 4's in-block iteration (VC_ITER_BLOCK: blocks of the states of h inner
    hosts, p local passes per global sweep, self-transitions solved) on the implicit form,
    several shapes, each device-timed to the same certified residual."""
    out = {"shapes": []}
    best = None
    for h, passes in ((0, 4), (1, 2), (1, 4), (1, 8)):
        try:
            mi.set_block_iteration(h, passes)
        except Exception:
            continue

        def solve():
            Vi.zero_()
            return mi.value_iterate(Vi, tol=args.tol, block=True)

        solve()
        t, (_, _, _, st) = _timed(torch, stream, solve, 3)
        row = {"inner_hosts": h, "block_states": mi.block_iteration_info()["block_states"], "passes": passes,
               "ms": t, "sweeps": int(st["sweeps"]), "ms_fp32_sweeps": st["ms_fp32"], "ms_fp64_refine": st["ms_fp64"],
               "us_per_sweep": 1e3 * st["ms_fp32"] / max(int(st["sweeps"]), 1), "certified": st["certified"] == 1}
        out["shapes"].append(row)
        if best is None or t < best["ms"]:
            best = row
    mi.set_block_iteration(-1, 4)
    out["best"] = best
    out["speedup_vs_self_loop"] = t_self_loop / best["ms"] if best else None
    return out


def variants(args, p, native, torch, dev, stream):
    """The other storage forms of the same workload, same step, device-timed."""
    out = {}
    forms = [("implicit", False, False)] + [(f, pd, sl) for sl in (False, True) for f in ("csr_f32", "csr_bf16")
                                             for pd in (False, True)]
    for form, padded, sliced in forms:
        if form == args.form and padded == args.padded and sliced == args.sliced:
            continue
        m = native.MDP.build(p, fmt=form, padded=padded, sliced=sliced)
        if form != "implicit":
            m.autotune(reps=5)
        info = m.info()
        V = torch.zeros(info["S"], dtype=torch.float32, device=dev)
        for _ in range(2):
            V.zero_()
            m.value_iterate(V, tol=args.tol)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        sweeps = 0
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            V.zero_()
            _, _, _, st = m.value_iterate(V, tol=args.tol)
            sweeps += st["sweeps"]
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps
        best = _best_plan(m) if form != "implicit" else None
        sweep_us = float(best.split()[-1]) if best else _sweep_us(m, torch, dev, stream)
        hbm = peaks()[0]
        alg = (8 * int(info["S"]) if form == "implicit" else
               algorithmic_sweep_bytes(int(info["S"]), int(info["A"]), int(info["nnz_logical"]), form == "csr_bf16"))
        out[form + ("+padded" if padded else "") + ("+sliced" if sliced else "")] = {
            "time_to_residual_ms": t, "updates_per_s": info["nnz_logical"] * sweeps / reps / (t / 1e3),
            "sweep_us": sweep_us,
            "sweep_alg_frac": alg / (sweep_us * 1e-6) / 1e9 / hbm,
            "sweep_stored_frac": info["sweep_bytes"] / (sweep_us * 1e-6) / 1e9 / hbm,
            "ncu_sol": implicit_sol() if form == "implicit" else None,
            "ms_fp32_sweeps": st["ms_fp32"], "ms_fp64_refine": st["ms_fp64"],
            "sweeps": sweeps // reps, "nnz_stored": int(info["nnz_stored"]),
            "nnz_sliced": int(info["nnz_sliced"]), "sweep_bytes": int(info["sweep_bytes"]),
            "tuned": best}
        m.close()
    return out


def _oracle_sweeps_threaded(p, nthreads: int, min_seconds: float):
    """Full Jacobi sweeps of the oracle (as it stands) with the state space split into
    nthreads contiguous ranges, one host thread each (the oracle's C routine runs outside
    the Python lock, so the threads run in parallel).  Returns (updates, seconds, sweeps)."""
    import threading

    import numpy as np

    import oracle

    S = oracle.num_states(p)
    V, Vn = np.zeros(S), np.zeros(S)
    bounds = [S * k // nthreads for k in range(nthreads + 1)]
    updates, sweeps = 0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < min_seconds and sweeps < 50:
        counts = [0] * nthreads

        def work(k):
            counts[k] = oracle.sweep_states(p, V, Vn, bounds[k], bounds[k + 1], 1)

        ts = [threading.Thread(target=work, args=(k,)) for k in range(nthreads)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        updates += sum(counts)
        V, Vn = Vn, V
        sweeps += 1
    return updates, time.perf_counter() - t0, sweeps


def cpu_baseline(p, args, min_seconds: float = 6.0):
    """The FP64 oracle's Bellman sweeps over the same instance: on every host core (the
    value) and on one thread (reported beside it)."""
    cores = os.cpu_count() or 1
    u1, t1, n1 = _oracle_sweeps_threaded(p, 1, min_seconds)
    un, tn, nn = _oracle_sweeps_threaded(p, cores, min_seconds)
    return {"value": un / tn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": u1 / t1,
            "sample": f"full Jacobi sweeps of the {args.workload} instance from V=0: {nn} sweep(s) on {cores} "
                      f"threads ({un} updates, {tn:.1f} s) and {n1} on one thread ({u1} updates, {t1:.1f} s)"}


# ------------------------------------------------------------------------ reference arm
def run_reference(args):
    import numpy as np

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2012_12419_gb300 import inputs

    import threading

    stride = 16  # one step: backups of every 16th state (1/16 of a sweep), on every host core
    cores = os.cpu_count() or 1
    if args.workload == "batched":
        # the 512 instances dealt round-robin to the cores; each core backs up every 16th
        # state of its instances
        ps = inputs.batch_params(512, seed=2)
        bufs = [(np.zeros(oracle.num_states(p)), np.zeros(oracle.num_states(p))) for p in ps]

        def part(k, c):
            return sum(oracle.sweep_states(ps[i], bufs[i][0], bufs[i][1], k % stride, oracle.num_states(ps[i]), stride)
                       for i in range(c, len(ps), cores))
    else:
        p = inputs.workload(args.workload)
        S = oracle.num_states(p)
        V = np.zeros(S)
        Vn = np.zeros(S)
        # contiguous state ranges aligned to the stride, one per core
        chunk = (S + cores - 1) // cores
        chunk = (chunk + stride - 1) // stride * stride

        def part(k, c):
            return oracle.sweep_states(p, V, Vn, c * chunk + k % stride, min(S, (c + 1) * chunk), stride)

    def one(k):
        counts = [0] * cores

        def work(c):
            counts[c] = part(k, c)

        ts = [threading.Thread(target=work, args=(c,)) for c in range(cores)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        return sum(counts)

    for k in range(max(3, args.warmup)):
        one(k)
    ups, secs = 0, 0.0
    for k in range(args.steps):
        t0 = time.perf_counter()
        ups += one(k)
        secs += time.perf_counter() - t0
    value = ups / secs
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "strong" if args.workload == "batched" else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": (step_config(args, oracle.csr_nnz(p), int(os.environ.get("WORLD_SIZE", "1")))
                   if args.workload != "batched" else {"workload": WORKLOAD_DESC[args.workload], "tol": args.tol}),
        "reference_form": f"FP64 oracle: successor enumeration and Jacobi backups on {cores} host threads",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: Jacobi backups of every {stride}th state of the "
                                   + ("512 instances" if args.workload == "batched" else "instance")
                                   + f", split over {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
