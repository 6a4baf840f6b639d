#!/usr/bin/env python
"""Benchmark of the LBM shape-optimisation hot path on GB300.

One benchmark step is one whole optimisation run on the 2048 x 1024
four-generation distributor tree (FP32 populations): reset to the initial
shape, solve 5000 time steps, then 50 times {exchange n_swap cells by the
optimality criterion, re-solve 5000 steps}; 51 x 5000 stream-collide sweeps
with the FP64 reductions of every solve.

Metric: fluid lattice updates per second (GLUPS), whole job.  `value` is
timed with CUDA events on the library's stream with the lattice resident in
device memory; `e2e` times the same run through the public API from a
pinned host cell map to the final cell map back on the host, creation and
destruction of the lattice included.  The roofline entry is the
stream-collide kernel: algorithmic bytes per launch (fluid cells x 72.125 B)
over its average launch time, measured with CUDA events inside the timed
region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With --impl reference the FP64 CPU oracle is timed on this host's cores on
a bounded sample of the same workload (the reference arm of this project).
Under torchrun (N > 1) every rank runs its own replica (seed = rank) and
value = updates of all ranks / slowest rank's time.
"""
import argparse
import json
import math
import os
import pathlib
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "D2Q9 fluid GLUPS (optimisation run, stream-collide + FP64 reductions + exchange)"
UNIT = "GLUPS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--iters", type=int, default=50, help="optimiser iterations per run")
    ap.add_argument("--lattice-steps", type=int, default=5000, help="time steps per solve")
    ap.add_argument("--precision", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-extras", action="store_true", help="skip the large-lattice and CPU legs")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--kernel-case", choices=["tree", "large"], default=None,
                    help="only create one lattice and run two 4-step solves (for ncu captures): "
                         "tree = 2048 x 1024 distributor, large = 8192 x 4096 channel array")
    return ap.parse_args()


def kernel_case(args):
    """Minimal run for a profiler: the stream-collide launches of the second
    solve are phase A then phase B of one plain pair."""
    import paper_1303_0107_gb300 as L
    from paper_1303_0107_gb300 import inputs as I
    prec = L.lib.PRECISIONS[args.precision]
    if args.kernel_case == "tree":
        cfg = I.config_tree_2048()
        cells, tau, u_max = cfg["cells"], cfg["tau"], cfg["u_max"]
    else:
        cells, tau, u_max = I.channel_array(8192, 4096, 16, fill=0.5), 0.6, 0.05
    lat = L.Lattice(cells, tau, u_max, precision=prec, residual_every=0)
    lat.solve(4)
    r = lat.solve(4)
    lat.close()
    print(json.dumps({"kernel_case": args.kernel_case, "precision": args.precision,
                      "fluid_cells": int((cells == 0).sum()), "dp": r["dp"]}))
    return 0


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled_traffic(kernel_file, name):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current kernel source (the summary records the source hash)."""
    import hashlib
    src = ROOT / "paper_1303_0107_gb300" / "csrc" / kernel_file
    summ = ROOT / "profiles" / name
    if not src.exists() or not summ.exists():
        return None
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    vals = {}
    for line in summ.read_text().splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip().lower()] = v.strip()
    if vals.get("source_sha256_16") != h:
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_workload"])
    except (KeyError, ValueError):
        return None


def oracle_rate(cells, tau, u_max, seconds):
    """Fluid updates per second of the FP64 oracle on a bounded sample."""
    import oracle as ora
    ny, nx = cells.shape
    p = ora.make_params(nx, ny, tau, 1.0, u_max)
    u_in = ora.inlet_profile(p, cells)
    f = ora.init(p, cells)
    fluid = int((cells == 0).sum())
    n = 2
    while True:  # calibrate: double the step count until a run takes 0.25 s
        t0 = time.perf_counter()
        f, *_ = ora.run(p, cells, u_in, f, n)
        t = time.perf_counter() - t0
        if t >= 0.25:
            break
        n *= 2
    n = max(2, int(seconds * n / t) // 2 * 2)
    t0 = time.perf_counter()
    ora.run(p, cells, u_in, f, n)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return fluid * n / dt, n, dt, cores


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle on the host cores, same workload and unit."""
    if rank != 0:
        return 0
    from paper_1303_0107_gb300 import inputs as I
    cfg = I.config_tree_2048(seed=0)
    for _ in range(args.warmup):
        oracle_rate(cfg["cells"], cfg["tau"], cfg["u_max"], 0.5)
    rates, total_updates, total_s = [], 0, 0.0
    for _ in range(args.steps):
        r, n, dt, cores = oracle_rate(cfg["cells"], cfg["tau"], cfg["u_max"], args.cpu_seconds / max(1, args.steps))
        rates.append(r)
        total_updates += r * dt
        total_s += dt
    value = total_updates / total_s / 1e9
    sample = (f"{cfg['name']}: {args.steps} samples of ~{args.cpu_seconds / max(1, args.steps):.1f} s "
              f"of FP64 time steps from rest (exchange and reductions excluded)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg["name"], "nx": cfg["nx"], "ny": cfg["ny"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.kernel_case:
        return kernel_case(args)

    import numpy as np
    import torch
    import paper_1303_0107_gb300 as L
    from paper_1303_0107_gb300 import inputs as I

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    prec = L.lib.PRECISIONS[args.precision]
    cfg = I.config_tree_2048(seed=rank)
    cells = cfg["cells"]
    fluid = int((cells == 0).sum())
    n_swap = max(1, int(0.002 * fluid))
    S, iters = args.lattice_steps, args.iters
    stream = torch.cuda.Stream()
    lat = L.Lattice(cells, cfg["tau"], cfg["u_max"], precision=prec, residual_every=100, stream=stream)

    def one_run(handle):
        handle.reset()
        r = handle.solve(S)
        dp0 = r["dp"]
        for _ in range(iters):
            r = handle.optimize_step(n_swap, S)
        return dp0, r

    for _ in range(args.warmup):
        one_run(lat)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    lat.kernel_time(reset=True)
    launches0 = L.kernel_launches()
    ev = []
    last = None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)  # evict the lattice from L2 between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        last = one_run(lat)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = L.kernel_launches() - launches0
    k_ms, k_launches, k_updates = lat.kernel_time()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    updates_per_step = fluid * S * (iters + 1)
    if dist is not None:
        t = torch.tensor([total_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = updates_per_step * args.steps * world / total_s / 1e9

    # roofline of the stream-collide kernel, from the timed region
    bpu = L.bytes_per_fluid_update(prec)
    avg_launch_s = (k_ms / 1e3) / max(k_launches, 1)
    bytes_per_launch = fluid * bpu
    achieved = bytes_per_launch / avg_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic("step.cu", "stream_collide_tree_2048x1024.md"),
                "peak_kind": peak_kind, "bytes_per_launch": bytes_per_launch,
                "avg_launch_us": avg_launch_s * 1e6,
                "note": "lattice working set (fluid cells) is L2-resident within a solve"}

    # end to end through the public API: pinned host cell map in, cell map out
    cells_pin = torch.from_numpy(cells).pin_memory()
    mask_out = torch.empty(cells.shape, dtype=torch.uint8).pin_memory()
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = L.Lattice(cells_pin.numpy(), cfg["tau"], cfg["u_max"], precision=prec, residual_every=100,
                      stream=stream)
        r = h.solve(S)
        for _ in range(iters):
            r = h.optimize_step(n_swap, S)
        h.read(L.FIELD_MASK, out=mask_out.numpy())
        h.close()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_times) / len(e2e_times)
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    sz = ctypes_sizes()
    n_out = r["n_outlets"]
    # host -> device: the cell map and parameters, plus the per-row inlet speeds,
    # outlet runs and lattice descriptors the library derives from them
    h2d = cells.nbytes + sz["params"] + 4 * cells.shape[0] + 8 * n_out + 3 * sz["view"]
    # device -> host: the reduction block of every solve, the exchange counters
    # of every iteration, the fluid counts, and the final cell map
    d2h = cells.nbytes + (iters + 1) * sz["result_block"] + iters * (32 + 8) + 8
    e2e = {"value": updates_per_step * world / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s}

    extras = {}
    if not args.no_extras and rank == 0:
        # beyond-L2 lattice: 8192 x 4096 array of 16 straight channels (~50 % fluid)
        big = I.channel_array(8192, 4096, 16, fill=0.5)
        bf = int((big == 0).sum())
        for pname, pv in (("f32", L.F32), ("bf16", L.BF16_SHIFTED)):
            hb = L.Lattice(big, 0.6, 0.05, precision=pv, residual_every=0, stream=stream)
            hb.solve(20)
            hb.kernel_time(reset=True)
            hb.solve(200)
            ms, nl, nu = hb.kernel_time()
            gbs = bf * L.bytes_per_fluid_update(pv) / ((ms / 1e3) / nl) / 1e9
            extras[f"large_8192x4096_{pname}"] = {"glups": nu / (ms / 1e3) / 1e9, "achieved_gbs": gbs,
                                                  "frac_of_measured_hbm": gbs / peak, "fluid_cells": bf}
            hb.close()
    cpu = None
    if not args.no_extras and rank == 0 and world == 1:
        r, n, dt, cores = oracle_rate(cells, cfg["tau"], cfg["u_max"], args.cpu_seconds)
        cpu = {"value": r / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{cfg['name']}: {n} FP64 time steps from rest, {dt:.1f} s"}

    if rank == 0:
        dp0, r_last = last
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == L.F32 else args.precision,
                "data": "synthetic",
                "config": {"workload": cfg["name"] + f"_{args.precision}_{iters + 1}x{S}", "nx": cfg["nx"],
                           "ny": cfg["ny"], "fluid_cells": fluid, "n_swap": n_swap,
                           "solves_per_step": iters + 1, "time_steps_per_solve": S,
                           "l2": "flushed between timed steps (256 MB write)",
                           "parallelism": f"replicas x{world}"},
                "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
                "cpu_baseline": cpu,
                "dense_glups": cfg["nx"] * cfg["ny"] * S * (iters + 1) * args.steps * world / total_s / 1e9,
                "dp_initial": dp0, "dp_final": r_last["dp"], "theta_final": r_last["theta"],
                "dg_final": r_last["dg"], "extras": extras}
        print(json.dumps(line))
    lat.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def ctypes_sizes():
    import ctypes
    from paper_1303_0107_gb300 import lib
    return {"params": ctypes.sizeof(lib.Params), "solve_result": ctypes.sizeof(lib.SolveResult),
            "opt_result": ctypes.sizeof(lib.OptResult), "view": 96, "result_block": 8 * (10 + lib.MAX_OUTLETS)}


if __name__ == "__main__":
    sys.exit(main())
