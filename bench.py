"""Benchmark: exact N-Queens counting on GB300 -- search nodes/s, solve time,
integer-roofline fraction.

One step = one pass of the whole device hot path over one batch: the persistent
search kernel over every subproblem of the N=18 board (per-prefix uint64 counts
written, weighted totals reduced per warp) with the prefixes already resident
in HBM. The end-to-end number (``e2e``) goes through the public C call
nq_total_ex: host enumeration, pinned host->device copy, search, device->host
read of the total, every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on
the host cores instead (a bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "search nodes/s and exact-count solve time at N=18/22 on 1 GB300; ALU roofline %"
UNIT = "nodes/s"
# 32-bit integer operations of the search per node (one queen placement):
# neg+and (lowest bit), xor (clear it), or (cols), or+shl (ld), or+shr (rd),
# nor3 (next row) -- the algorithmic work of Algorithm 2's loop body.
ALU_OPS_PER_NODE = 10
# 32-bit integer ALU lanes per clock per SM the roofline is drawn against
# (measured issue rate of the ALU pipe; see nq_probe_alu and the design notes).
ALU_LANES_PER_CLK_SM = 64
SM_MAX_MHZ_FALLBACK = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=18)
    ap.add_argument("--d", type=int, default=0, help="prefix depth (0 = library default)")
    ap.add_argument("--layout", default="default", choices=["default", "paper", "reg", "wt", "wt32", "wt32a", "wtm",
                                                      "regm"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--bps", type=int, default=0, help="blocks per SM (0 = max)")
    ap.add_argument("--order", type=int, default=0, help="0 default, 1 index order, 2 reverse")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# --- distributed plumbing (one process per GPU; replicas, weak scaling) -------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world):
    if world <= 1:
        return None
    import torch.distributed as dist
    backend = "nccl" if __import__("torch").cuda.is_available() else "gloo"
    dist.init_process_group(backend=backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, device) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --- clocks sampled during the timed region ---------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                "power_w_max": max(power) if power else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# --- CPU oracle baseline --------------------------------------------------------

def oracle_rate(n: int, d: int, seconds: float, seed: int = 7) -> dict:
    """The CPU oracle (all host cores, dynamic pulling) on a seeded sample of the
    same workload's subproblems, grown until it has run about `seconds`."""
    import oracle
    oracle.build()
    cols, _ = oracle.prefixes(n, d)
    rng_order = np.random.default_rng(seed).permutation(len(cols))  # seeded, no repeats
    done_nodes, done = 0, 0
    chunk = 64
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and done < len(rng_order):
        idx = rng_order[done:done + chunk]
        _, nodes = oracle.count_prefixes(n, cols[idx])
        done_nodes += int(nodes.sum())
        done += len(idx)
        chunk = min(chunk * 2, 65536)
    dt = time.perf_counter() - t0
    return {"value": done_nodes / dt, "unit": UNIT, "cores": oracle.default_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": f"{done} seeded-random subproblems of N={n}, d={d} ({done_nodes} nodes)"}


def run_reference(args):
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
        return
    n = args.n
    from paper_2511_12009_gb300 import nq  # only for the workload's depth
    d = args.d or nq.default_depth(n)
    per_step = max(1.0, min(8.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate(n, d, per_step / 4, seed=1)
    rates, total_nodes, total_s = [], 0, 0.0
    for k in range(args.steps):
        r = oracle_rate(n, d, per_step, seed=100 + k)
        rates.append(r)
        total_nodes += r["value"] * r["seconds"]
        total_s += r["seconds"]
    value = total_nodes / total_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": f"N={n} full count, d={d} prefixes", "n": n,
                                            "d": d},
            "cpu_baseline": {"kind": "oracle", "cores": rates[0]["cores"], "value": value,
                             "unit": UNIT,
                             "sample": f"each step: seeded-random subproblems of N={n}, d={d} "
                                       f"for ~{per_step:.0f} s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --- our arm ---------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2511_12009_gb300 import nq

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = dist_init(world)
    lib = nq.lib()
    del lib
    n = args.n
    d = args.d or nq.default_depth(n)
    cfg = nq.make_config(args.layout, args.block, args.bps, args.order, d)
    stream = torch.cuda.Stream(device)

    # inputs resident in HBM
    pre_h = nq.enumerate_prefixes(n, d)
    pre = nq.to_device(pre_h, device)
    m = len(pre_h)
    counts = torch.zeros(m, dtype=torch.int64, device=device)
    totals = torch.zeros(32, dtype=torch.int64, device=device)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=device)

    # nodes of this workload: the diagnostic build counts them once, untimed
    nodes_t = torch.zeros(m, dtype=torch.int64, device=device)
    with torch.cuda.stream(stream):
        totals.zero_()
        nq.count_ex(pre, d, n, counts, nodes_t, totals, cfg, stream)
    nq.sync(stream)
    nodes_per_step = int(nodes_t.cpu().numpy().view(np.uint64).sum())
    total_q = int(totals.cpu().numpy().view(np.uint64)[n])
    del nodes_t

    def step():
        totals.zero_()
        nq.count_ex(pre, d, n, counts, None, totals, cfg, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    nq.sync(stream)
    if int(totals.cpu().numpy().view(np.uint64)[n]) != total_q:
        raise SystemExit("warm-up total differs from the first run")

    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(dist)
    torch.cuda.synchronize(device)
    clocks.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()  # L2 (129 MB) flushed between steps, outside the timed events
            starts[k].record(stream)
            step()
            ends[k].record(stream)
    torch.cuda.synchronize(device)
    t_wall = time.perf_counter() - t_wall0
    barrier(dist)
    clk = clocks.stop()
    rc = nq.lib().nq_sync(stream.cuda_stream)
    if rc != 0:
        raise SystemExit(f"search reported {nq.strerror(rc)}")
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_s = sum(step_ms) * 1e-3
    kern_s_max = max_over_ranks(dist, kern_s, device)
    if int(totals.cpu().numpy().view(np.uint64)[n]) != total_q:
        raise SystemExit("timed total differs from the first run")
    value = nodes_per_step * args.steps * world / kern_s_max
    ms_per_step = 1e3 * kern_s_max / args.steps

    # end to end through the public C call (enumerate, H2D, search, D2H)
    e2e = None
    if args.e2e_steps > 0:
        e2e_times = []
        e2e_cfg = nq.make_config(args.layout, args.block, args.bps, args.order, d)
        for k in range(args.e2e_steps + 1):
            t0 = time.perf_counter()
            r = nq.total_ex(n, e2e_cfg)
            dt = time.perf_counter() - t0
            if r["total"] != total_q:
                raise SystemExit("end-to-end total differs")
            if k:  # the first call warms the pinned staging buffer
                e2e_times.append(dt)
        e2e_s = max_over_ranks(dist, float(np.mean(e2e_times)), device)
        e2e = {"value": nodes_per_step * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": m * 16, "d2h_bytes_per_step": 8,
               "solve_ms": 1e3 * e2e_s, "enumerate_ms": r["enumerate_ms"],
               "upload_ms": r["upload_ms"]}

    # roofline of the one kernel: algorithmic int ops per launch / launch time
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or SM_MAX_MHZ_FALLBACK)
    peak_tops = sms * sm_max * 1e6 * ALU_LANES_PER_CLK_SM / 1e12
    achieved_tops = nodes_per_step * ALU_OPS_PER_NODE / (kern_s_max / args.steps) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s",
                "frac": achieved_tops / peak_tops, "traffic": None,
                "ops_per_node": ALU_OPS_PER_NODE, "nodes_per_launch": nodes_per_step,
                "peak_basis": f"{sms} SMs x {sm_max:.0f} MHz x {ALU_LANES_PER_CLK_SM} int32 ALU "
                              f"lanes/clk/SM"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_rate(n, d, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": {"workload": f"N={n} full count, d={d} prefixes ({m} subproblems)",
                           "n": n, "d": d, "subproblems": m, "nodes_per_step": nodes_per_step,
                           "layout": args.layout, "block": args.block, "blocks_per_sm": args.bps,
                           "order": args.order,
                           "l2": "flushed between steps (256 MiB write outside the timed events)",
                           "parallelism": f"replicas x{world}"},
                "solve_ms": ms_per_step, "total": total_q, "wall_s": t_wall,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": args.steps}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
