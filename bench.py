"""Benchmark: minimum spanning tree throughput on one GB300 (or N replicas).

Default workload (the headline): the 1024 x 1024 four-neighbour grid
(n = 1,048,576, m = 2,095,104), uint32 weights a random permutation of 1..m,
edge order shuffled.  One step = one full solve (init, every Boruvka round,
emit) with the inputs already resident in HBM.  The 25 MB input fits in the
129 MB L2, so L2 is flushed (a 256 MiB write) between timed steps, outside
the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config 1|2|3] [--no-cpu-baseline]

Under torchrun (N > 1) every rank solves its own replica of the workload (a
single solve does not shard); value = edges of all ranks / max rank time.
--impl reference times the CPU oracle (Kruskal, one thread) on the same
workload, rank 0 only.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MST Medges/s and HBM roofline fraction; batched graphs/s with p50/p99 latency"
UNIT = "Medges/s"
L2_FLUSH_BYTES = 256 << 20


def workload(cfg: int):
    from paper_2005_06913_gb300 import graphgen as gg
    g = gg.config(cfg)
    names = {1: "C1 random connected n=4096 m=32768",
             2: "C2 grid2d 1024x1024 (4-neighbour), shuffled edge order",
             3: "C3 R-MAT scale 22 edge factor 8, connected"}
    return g, names[cfg]


def traffic_for(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/ncu_traffic.txt: "kernel source_sha256 bytes_per_launch"),
    or None when absent or taken on different kernel source."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    src = os.path.join(ROOT, "paper_2005_06913_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(src)):
        h.update(open(os.path.join(src, f), "rb").read())
    sha = h.hexdigest()[:16]
    for line in open(p):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[1] == sha:
            return float(f[2])
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi (every 50 ms)
    from before warm-up to after the timed region; summary() keeps the
    samples taken inside the timed window (or, when the window is shorter
    than the sampling period, the samples around it, and says so)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.window = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            deadline = time.time() + 5
            while time.time() < deadline and os.path.getsize(self.path) == 0:
                time.sleep(0.05)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        import datetime
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), [x.lower() == "active" for x in f[6:10]]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        t0, t1 = self.window or (rows[0][0], rows[-1][0])
        inside = [r for r in rows if t0 <= r[0] <= t1]
        where = "inside the timed region"
        if not inside:  # region shorter than the sampling period
            inside = sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:3]
            where = "nearest to a timed region shorter than the 50 ms sampling period"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[3][i]})
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside), "reasons": reasons,
                "samples": len(inside), "where": where}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(g, budget_s: float = 12.0):
    """The oracle (Kruskal, one thread) on the full workload, repeated until
    about budget_s seconds of CPU work; Medges/s."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.kruskal(g.n, g.src, g.dst, g.w)
        reps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": g.m * reps / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle Kruskal (oracle/mst_oracle.c, 1 thread) on the full workload "
                      f"(m={g.m}), {reps} solves in {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    g, wname = workload(args.config)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.kruskal(g.n, g.src, g.dst, g.w)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.kruskal(g.n, g.src, g.dst, g.w)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = g.m * args.steps / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wname, "n": g.n, "m": g.m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: oracle Kruskal (1 thread) on the full workload (m={g.m})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_e2e(B, h, g, ws, stream, args):
    """Same metric through mst_solve_host: pinned host inputs copied in and
    the tree copied out inside every timed step."""
    import torch
    hs = torch.from_numpy(g.src).pin_memory()
    hd = torch.from_numpy(g.dst).pin_memory()
    hw = torch.from_numpy(g.w.view(np.int32)).pin_memory()
    ho = torch.empty(max(g.n - 1, 1), dtype=torch.int32).pin_memory()
    hc = torch.zeros(1, dtype=torch.int64).pin_memory()
    for _ in range(2):
        B.mst_solve_host(h, B.MST_W_U32, g.n, g.m, hs, hd, hw, ho, hc, stream)
    steps = max(3, min(args.steps, 50))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        st = B.mst_solve_host(h, B.MST_W_U32, g.n, g.m, hs, hd, hw, ho, hc, stream)
        if st != B.MST_OK:
            raise B.MstError(st, "mst_solve_host")
    dt = (time.perf_counter() - t0) / steps
    if int(hc.item()) != g.n - 1:
        raise RuntimeError("e2e self-check failed")
    return {"value": ws * g.m / dt / 1e6, "unit": UNIT,
            "h2d_bytes_per_step": 12 * g.m, "d2h_bytes_per_step": 4 * (g.n - 1) + 8,
            "ms_per_step": dt * 1e3, "steps": steps,
            "timer": "host wall clock around the blocking mst_solve_host call"}


def run_ours(args):
    import torch

    from paper_2005_06913_gb300 import binding as B
    from paper_2005_06913_gb300 import build as build_mod

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    if rank == 0:
        build_mod.build()
    if dist is not None:
        dist.barrier()
    g, wname = workload(args.config)
    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    w = torch.from_numpy(g.w.view(np.int32)).cuda()
    out = torch.empty(max(g.n - 1, 1), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    h = B.mst_create(dev, 0)
    B.mst_set_single_schedule(h, 1 if args.schedule == "fused" else 2, 0)

    def solve():
        st = B.mst_solve(h, g.n, g.m, src, dst, w, out, cnt, stream)
        if st != B.MST_OK:
            raise B.MstError(st, "mst_solve")

    for _ in range(max(args.warmup, 3)):
        solve()
    status = B.mst_get_status(h, stream)
    if status != B.MST_OK or int(cnt.item()) != g.n - 1:
        raise RuntimeError(f"self-check failed: status {B.mst_status_string(status)}, "
                           f"count {int(cnt.item())} != {g.n - 1}")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clk = ClockSampler(dev).start()
    for _ in range(3):
        solve()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    for k in range(args.steps):
        if not args.no_flush:
            flush.fill_(k)  # evict the inputs from L2 (untimed)
        starts[k].record(stream)
        solve()
        ends[k].record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    clk.mark(t_wall0, t_wall1)
    clk.stop()
    t_wall = t_wall1 - t_wall0
    if dist is not None:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    if dist is not None:
        tt = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    status = B.mst_get_status(h, stream)
    clocks = clk.summary()
    rounds_e, rounds_v = B.mst_get_round_stats(h, stream)

    # per-phase times of the timed kernel (fused schedule: its own phase log)
    prof = B.mst_profile_last_solve(h, stream)
    hbm_peak, peak_kind = peaks()
    solve_bytes = sum(p["alg_bytes"] for p in prof)
    step_s = total_ms / args.steps * 1e-3
    kernels = [{"name": p["name"], "count": p["launches"], "ms": round(p["total_ms"], 4),
                "alg_MB": round(p["alg_bytes"] / 1e6, 3),
                "GBps": round(p["alg_bytes"] / max(p["total_ms"], 1e-9) / 1e6, 1)} for p in prof]
    if args.schedule == "fused":
        launches_per_step = 1
        dom_name, dom_bytes, dom_s, dom_launches = "k_solve", solve_bytes, step_s, 1
    else:
        launches_per_step = sum(p["launches"] for p in prof)
        dom = max(prof, key=lambda p: p["total_ms"])
        dom_name, dom_bytes, dom_s, dom_launches = (dom["name"], dom["alg_bytes"],
                                                    dom["total_ms"] * 1e-3, dom["launches"])
    achieved = dom_bytes / dom_s / 1e9
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic_for(dom_name),
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy)",
                "launches_per_step": dom_launches,
                "alg_bytes_per_launch": dom_bytes / max(dom_launches, 1),
                "duration_source": "CUDA events per step (whole solve)" if args.schedule == "fused"
                else "CUDA-event replay of each kernel"}

    # end to end through the host-buffer C-ABI call, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(B, h, g, ws, stream, args)
    line = {
        "metric": METRIC, "value": ws * g.m * args.steps / (total_ms * 1e-3) / 1e6, "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wname, "n": g.n, "m": g.m, "rounds": len(rounds_e) - 1,
                   "live_edges_per_round": rounds_e, "components_per_round": rounds_v,
                   "l2": "flushed between timed steps (256 MiB write, outside the timed events)"
                         if not args.no_flush else "not flushed",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "timer": "CUDA events per step on the launching stream"},
        "roofline": roofline,
        "phases" if args.schedule == "fused" else "kernel_replay": kernels,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
        "device_status": B.mst_status_string(status),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g)
    B.mst_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3])
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--schedule", choices=["fused", "graph"], default="fused")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
