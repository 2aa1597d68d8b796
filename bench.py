#!/usr/bin/env python3
"""Throughput of the F.A.S.T. time step on GB300 (one JSON line on rank 0).

A timed "step" is one full time step of the model -- planning (FP32 weights
with FP64 re-check of draws near a boundary) followed by the sequential
movement phase, emulated in rounds -- over the precision workload: a
4000x4000 grid with 10% obstacles, 16 exits, 1,000,000 agents clustered by a
32-component Gaussian mixture, v_m = 4, k_S = 1.2.

  value        agent-steps/s of the whole job, summed CUDA-event times of the
               K timed steps (L2 flushed by a 512 MiB write before each step,
               outside the events), max over ranks
  choices_per_s  desired-cell choices/s of the planning phase alone
  fp64_form    the same with every agent planned by the all-FP64 kernel
  e2e          agent-steps/s through the public API with host buffers: each
               step places the state from pinned host memory, steps once and
               reads cells and desired cells back
  roofline     the dominant kernel (movement rounds): algorithmic bytes per
               launch / its average event time, against the measured HBM copy
               bandwidth; roofline_plan the same for the planning kernel
  cpu_baseline the FP64 CPU oracle on this host's cores (rank 0, N=1)

--impl reference times the CPU oracle alone (planning loop with the paper's
OpenMP partition over all host cores, sequential movement) on the same
workload, metric and unit.

Multi-GPU: one process per GPU; every rank simulates its own replicate (seed
+ rank) with no collective on the data path ("scaling": "weak").
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
sys.path.insert(0, ROOT)

METRIC = "desired-cell choices/s and agent-steps/s at v_m=4, FP32+recheck vs FP64 form"
UNIT = "agent-steps/s"
L2_FLUSH_BYTES = 512 << 20

# Sources each profiled kernel is compiled from; a committed ncu summary's
# DRAM traffic is reported only while these files are unchanged.
KERNEL_SOURCES = {
    "k_plan_tile": ["plan_kernels.cuh", "fast_device.cuh", "fast_internal.h"],
    "k_move_rounds": ["move.cu", "fast_device.cuh", "fast_internal.h"],
}


def source_digest(kernel):
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_0911_2900_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload_name):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from the
    committed ncu summary of this kernel on this workload, or None when there
    is none or the kernel's sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload_name}.md")
    try:
        fields = {}
        with open(path) as fh:
            for ln in fh:
                if ":" in ln and ln.split(":")[0] in ("source_digest", "dram_bytes_per_launch"):
                    k, v = ln.split(":", 1)
                    fields[k] = v.strip()
        if fields.get("source_digest") != source_digest(kernel):
            return None
        return float(fields["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="precision",
                   choices=["precision", "room", "corridors", "stress"])
    p.add_argument("--fp64-steps", type=int, default=3)
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--cpu-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--json-out", default=None)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(name, rank):
    from paper_0911_2900_gb300 import workloads as wl

    if name == "precision":
        return wl.config_precision(seed=rank)
    if name == "room":
        return wl.config_small_room(seed=rank)
    if name == "corridors":
        return wl.config_corridors(v_m=4, seed=rank)
    return wl.config_stress(seed=rank)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
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
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, world, op="max"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def plan_bytes(n_agents, union_cells, mask_words):
    """Algorithmic bytes of one planning pass: per agent id, cell, mask,
    desired write and own-record write; per cell of the reach union one
    4-byte record."""
    return n_agents * (4 + 4 + 8 * mask_words + 4 + 4) + union_cells * 4


def move_bytes(movers, footprint_cells):
    """Algorithmic bytes of one movement phase: every mover reads its start
    cell and desired cell (8 B) and the records of its footprint (4 B each),
    and writes two cell records and its new cell (12 B)."""
    return movers * (8 + 12) + footprint_cells * 4


def cpu_oracle_rate(w, steps, threads):
    import oracle

    sim = oracle.Sim(w.cell_type, v=w.v_m, kS=w.k_S, seed=w.seed)
    sim.place(w.cells)
    r = sim.run(0, steps, threads=threads, digests=False)
    agent_steps = int(len(w.cells)) + int(r["alive"][:-1].sum()) if steps > 1 else len(w.cells)
    plan_s, move_s = r["plan_s"], r["move_s"]
    return dict(agent_steps=agent_steps, plan_s=plan_s, move_s=move_s,
                value=agent_steps / (plan_s + move_s),
                choices_per_s=agent_steps / plan_s)


def bench_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = make_workload(args.workload, 0)
    threads = os.cpu_count() or 1
    import oracle

    sim = oracle.Sim(w.cell_type, v=w.v_m, kS=w.k_S, seed=w.seed)
    sim.place(w.cells)
    if args.warmup:
        sim.run(0, args.warmup, threads=threads, digests=False)
    alive0 = int((sim.cell >= 0).sum())
    t0 = time.perf_counter()
    r = sim.run(args.warmup, args.steps, threads=threads, digests=False)
    wall = time.perf_counter() - t0
    agent_steps = alive0 + int(r["alive"][:-1].sum())
    value = agent_steps / (r["plan_s"] + r["move_s"])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * (r["plan_s"] + r["move_s"]) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "grid": f"{w.shape[1]}x{w.shape[0]}",
                   "agents": int(len(w.cells)), "v_m": w.v_m, "k_S": w.k_S,
                   "precision": "fp64 (CPU oracle)"},
        "choices_per_s": agent_steps / r["plan_s"],
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} full steps of {w.name} after {args.warmup} "
                                   f"warm-up steps; planning on {threads} threads with the "
                                   f"paper's OpenMP partition, movement serial"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_ours(args):
    import numpy as np
    import torch

    import paper_0911_2900_gb300 as fg

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    w = make_workload(args.workload, rank)
    n0 = int(len(w.cells))
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def timed_steps(ctx, k, record_phases=True):
        step_ms, phases = [], []
        for i in range(k):
            flush.fill_(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.step(1)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            if record_phases:
                phases.append(ctx.phase_times())
        return step_ms, phases

    # ---- FP32 + FP64 re-check -------------------------------------------------
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    ctx.step(args.warmup)
    torch.cuda.synchronize()
    u0 = ctx.reach_union(0)
    _, _, st0 = ctx.readback(0, 0)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    clocks = Clocks(gpu_index)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    step_ms, phases = timed_steps(ctx, args.steps)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    _, _, st1 = ctx.readback(0, 0)
    mv_wait, mv_us = ctx.move_profile()
    u1 = ctx.reach_union(0)
    agent_steps = st1["agent_steps"] - st0["agent_steps"]
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    T = sum(step_ms) / 1e3
    plan_ms = [p[0] for p in phases]
    recheck_ms = [p[1] for p in phases]
    prep_ms = [p[2] for p in phases]
    rounds_ms = [p[3] for p in phases]
    other_ms = [p[4] for p in phases]
    T_max = max_over_ranks(T, world)
    total_agent_steps = max_over_ranks(agent_steps, world, op="sum")
    value = total_agent_steps / T_max
    choices = total_agent_steps / max_over_ranks((sum(plan_ms) + sum(recheck_ms)) / 1e3, world)
    n_avg = agent_steps / args.steps
    mw = 1 if w.v_m <= 4 else 2
    bytes_plan = plan_bytes(n_avg, 0.5 * (u0 + u1), mw)
    mean_plan_s = statistics.mean(plan_ms) / 1e3
    peak, peak_kind = measured_peaks()
    achieved = bytes_plan / mean_plan_s / 1e9
    movers = (st1["movers"] - st0["movers"]) / args.steps
    foot = (st1["footprint_cells"] - st0["footprint_cells"]) / args.steps
    bytes_move = move_bytes(movers, foot)
    mean_rounds_s = statistics.mean(rounds_ms) / 1e3
    achieved_move = bytes_move / mean_rounds_s / 1e9

    # ---- the all-FP64 form ------------------------------------------------------
    ctx64 = fg.Context(1, "fp64")
    ctx64.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx64.place(0, w.cells)
    ctx64.step(1)
    torch.cuda.synchronize()
    _, _, s640 = ctx64.readback(0, 0)
    ms64, ph64 = timed_steps(ctx64, args.fp64_steps)
    _, _, s641 = ctx64.readback(0, 0)
    as64 = s641["agent_steps"] - s640["agent_steps"]
    fp64_value = max_over_ranks(as64, world, "sum") / max_over_ranks(sum(ms64) / 1e3, world)
    fp64_choices = max_over_ranks(as64, world, "sum") / max_over_ranks(
        sum(p[0] + p[1] for p in ph64) / 1e3, world)
    ctx64.close()

    # ---- end to end through the public API with host buffers ---------------------
    cells_d, _, st = ctx.readback(0, n0)
    alive_ids = np.flatnonzero(cells_d >= 0).astype(np.int32)
    n_alive = len(alive_ids)
    h_cells = torch.empty(n_alive, dtype=torch.int32, pin_memory=True).numpy()
    h_ids = torch.empty(n_alive, dtype=torch.int32, pin_memory=True).numpy()
    out_cells = torch.empty(n0, dtype=torch.int32, pin_memory=True).numpy()
    out_des = torch.empty(n0, dtype=torch.int32, pin_memory=True).numpy()
    h_cells[:] = cells_d[alive_ids]
    h_ids[:] = alive_ids
    t_step = st["step"]
    e2e_agent_steps = 0
    barrier()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter()
    for i in range(args.e2e_steps):
        ctx.place(0, h_cells, ids=h_ids, start_step=t_step)
        ctx.step(1)
        ctx.readback(0, n0, cells_out=out_cells, desired_out=out_des)
        e2e_agent_steps += len(h_cells)
        keep = out_cells[h_ids] >= 0
        h_ids_new = h_ids[keep]
        h_cells_new = out_cells[h_ids_new]
        h_cells = h_cells[:len(h_ids_new)]
        h_ids = h_ids[:len(h_ids_new)]
        h_cells[:] = h_cells_new
        h_ids[:] = h_ids_new
        t_step += 1
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t_e2e
    barrier()
    e2e_value = max_over_ranks(e2e_agent_steps, world, "sum") / max_over_ranks(t_e2e, world)
    ctx.close()

    # ---- CPU baseline (the oracle), rank 0 at N = 1 ------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        c = cpu_oracle_rate(w, args.cpu_steps, threads)
        cpu = {"value": c["value"], "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {args.cpu_steps} steps of {w.name} ({n0} agents); planning "
                         f"on {threads} threads (paper's OpenMP partition), movement serial",
               "choices_per_s": c["choices_per_s"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * T_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "grid": f"{w.shape[1]}x{w.shape[0]}",
                       "agents": n0, "v_m": w.v_m, "k_S": w.k_S, "reach": "l2",
                       "precision": "fp32 weights + fp64 re-check",
                       "l2": "flushed before every timed step (512 MiB write, outside events)",
                       "parallelism": f"replicas x{world}"},
            "choices_per_s": choices,
            "fp64_form": {"value": fp64_value, "choices_per_s": fp64_choices, "unit": UNIT,
                          "steps": args.fp64_steps},
            "speedup_vs_fp64_form": value / fp64_value,
            "phase_ms": {"plan": statistics.mean(plan_ms), "recheck": statistics.mean(recheck_ms),
                         "move_prep": statistics.mean(prep_ms),
                         "move_rounds": statistics.mean(rounds_ms),
                         "other": statistics.mean(other_ms)},
            "movers_per_step": movers,
            "rechecked_per_step": (st1["rechecked"] - st0["rechecked"]) / args.steps,
            "tile_fallback_warps_per_step": (st1["tile_fallbacks"] - st0["tile_fallbacks"]) / args.steps,
            "move_rounds_per_step": (st1["move_rounds"] - st0["move_rounds"]) / args.steps,
            "move_last_step": {"waiting_after_round": [int(x) for x in mv_wait[:12]],
                               "round_us": [round(float(x), 2) for x in mv_us[:12]],
                               "rounds": int(len(mv_wait)),
                               "phases_max_over_blocks": [round(float(x) / 1e3, 2) if i not in (4, 5) else int(x)
                                                          for i, x in enumerate(ctx.last_move_phases)]},
            "roofline": {"bound": "hbm", "kernel": "k_move_rounds", "achieved": achieved_move,
                         "peak": peak, "unit": "GB/s", "frac": achieved_move / peak,
                         "traffic": measured_traffic("k_move_rounds", w.name),
                         "peak_kind": peak_kind, "bytes_per_launch": bytes_move,
                         "note": "dominant kernel; bound by the number of rounds and "
                                 "dependent scattered memory operations, not bandwidth"},
            "roofline_plan": {"bound": "hbm", "kernel": "k_plan_tile", "achieved": achieved,
                              "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                              "traffic": measured_traffic("k_plan_tile", w.name),
                              "peak_kind": peak_kind, "bytes_per_launch": bytes_plan,
                              "union_cells": 0.5 * (u0 + u1)},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * n_alive, "d2h_bytes_per_step": 8 * n0},
            "gpu_launches": int(launches),
            "clocks": clk,
            "wall_s_timed": t_wall,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        s = json.dumps(line)
        print(s, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(s + "\n")
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return bench_reference(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
