#!/usr/bin/env python
"""Benchmark of the LBM shape-optimisation hot path on GB300.

One benchmark step is one whole optimisation run on the 2048 x 1024
four-generation distributor tree (FP32 populations): reset to the initial
shape, solve 100 000 time steps (the converged flow field of Sec. 2.3 step
2: the residual falls to ~2e-5), then 50 times {exchange n_swap = 319 cells
by the optimality criterion, re-solve 5000 steps}; 350 000 stream-collide
sweeps with the FP64 reductions of every solve.  From the converged start
the pressure drop falls at every iteration (0.0275 -> 0.0097 measured).

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
    from paper_1303_0107_gb300 import inputs as I
    tree = I.load_config("tree_2048x1024_g4")
    served = I.load_config("served_poisson_200")
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--iters", type=int, default=tree["n_iter"], help="optimiser iterations per run")
    ap.add_argument("--lattice-steps", type=int, default=tree["steps"], help="time steps per re-solve")
    ap.add_argument("--first-steps", type=int, default=tree["first_solve_steps"],
                    help="time steps of the first solve (run to a converged flow field)")
    ap.add_argument("--precision", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-extras", action="store_true", help="skip every leg after the main run")
    ap.add_argument("--legs", default="large,tjunction,precision,models,collector,d3q19,batched,served",
                    help="legs after the main run: large (8192 x 4096 lattice), precision (BF16/FP16 vs the "
                         "FP64 oracle; also the CPU baseline), tjunction (128 x 64 T, launch-bound), "
                         "models (collision models on the tree), "
                         "collector (the paper's half-domain collector, 151 optimisation steps), "
                         "d3q19 (the D3Q19 path: step rates, optimisation loop, oracle rate), "
                         "batched (256 candidates), served (request loop), "
                         "sweep (served at 50, 100, 200 and 400 requests/s, 10 s each; not in the default run)")
    ap.add_argument("--serve-rate", type=float, default=served["rate_per_s"],
                    help="served leg: Poisson arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=served["seconds"], help="served leg: arrival window")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--log", default=None,
                    help="write one JSON line per solve of the timed runs (run, iteration, dp, m_in, residual, "
                         "theta, D_g, outlet flow rates, fluid cells, exchanged cells, time) to this file")
    ap.add_argument("--kernel-case", choices=["tree", "large", "batch", "tree3d", "duct3d"], default=None,
                    help="only create one lattice and run two solves of --kernel-steps steps (for ncu "
                         "captures): tree = 2048 x 1024 distributor, large = 8192 x 4096 channel array, "
                         "batch = the 256 candidate distributors in one batch, "
                         "tree3d = 384 x 192 x 192 D3Q19 distributor, duct3d = 256 x 128 x 128 D3Q19 duct")
    ap.add_argument("--kernel-steps", type=int, default=4)
    ap.add_argument("--kernel-cpt", type=int, default=0,
                    help="kernel case (2D): run with this many cells per thread (0: the tuner's choice)")
    ap.add_argument("--kernel-resident", action="store_true",
                    help="kernel case (2D): on-chip resident steps (one launch per solve)")
    ap.add_argument("--kernel-paired", action="store_true",
                    help="kernel case (2D, batch): paired tasks (interior 64-cell windows two cells a lane)")
    ap.add_argument("--kernel-cells", action="store_true",
                    help="kernel case (2D, batch): compacted fluid-cell tasks (32 consecutive fluid cells a warp)")
    ap.add_argument("--kernel-wpb", type=int, default=8, help="kernel case: warps per block of a fixed shape")
    ap.add_argument("--kernel-stages", type=int, default=0,
                    help="kernel case, paired or cell tasks: populations copied into shared memory this many "
                         "tasks ahead")
    return ap.parse_args()


def kernel_case(args):
    """Minimal run for a profiler: the stream-collide launches of the second
    solve are phase A then phase B of one plain pair."""
    import paper_1303_0107_gb300 as L
    from paper_1303_0107_gb300 import inputs as I
    prec = L.lib.PRECISIONS[args.precision]
    if args.kernel_case in ("tree3d", "duct3d"):
        if args.kernel_case == "tree3d":
            cfg = I.config_tree3d()
            cells, tau, u_max = cfg["cells"], cfg["tau"], cfg["u_max"]
        else:
            cells, tau, u_max = I.duct3d(256, 126, 126), 0.6, 0.05
        lat = L.Lattice3(cells, tau, u_max, precision=prec)
        lat.solve(args.kernel_steps)
        r = lat.solve(args.kernel_steps)
        lat.close()
        print(json.dumps({"kernel_case": args.kernel_case, "precision": args.precision,
                          "fluid_cells": int((cells == 0).sum()), "dp": r["dp"]}))
        return 0
    if args.kernel_case == "batch":
        cands = I.config_candidates(256)
        b = L.Batch([dict(cells=c["cells"], tau=c["tau"], u_max=c["u_max"]) for c in cands], precision=prec,
                    residual_every=0)
        if args.kernel_paired:
            b.set_step_config(args.kernel_wpb, persistent=4, cells_per_thread=2, stages=args.kernel_stages)
        elif args.kernel_cells:
            b.set_step_config(args.kernel_wpb, persistent=3, stages=args.kernel_stages)
        b.solve(args.kernel_steps)
        r = b.solve(args.kernel_steps)
        shape = b.step_config()
        b.close()
        print(json.dumps({"kernel_case": "batch", "precision": args.precision,
                          "fluid_cells": sum(int((c["cells"] == 0).sum()) for c in cands), "dp0": r[0]["dp"],
                          "step_config": list(shape)}))
        return 0
    if args.kernel_case == "tree":
        cfg = I.config_tree_2048()
        cells, tau, u_max = cfg["cells"], cfg["tau"], cfg["u_max"]
    else:
        cells, tau, u_max = I.channel_array(8192, 4096, 16, fill=0.5), 0.6, 0.05
    lat = L.Lattice(cells, tau, u_max, precision=prec, residual_every=0)
    if args.kernel_resident:
        lat.set_step_config(8, persistent=2)
    elif args.kernel_paired:
        lat.set_step_config(args.kernel_wpb, persistent=4, cells_per_thread=2, stages=args.kernel_stages)
    elif args.kernel_cpt:
        lat.set_step_config(8, cells_per_thread=args.kernel_cpt)
    lat.solve(args.kernel_steps)
    r = lat.solve(args.kernel_steps)
    shape = lat.step_config()
    lat.close()
    print(json.dumps({"kernel_case": args.kernel_case, "precision": args.precision,
                      "fluid_cells": int((cells == 0).sum()), "dp": r["dp"], "step_config": list(shape)}))
    return 0


def max_over_ranks(value, dist, device):
    """The largest value over all ranks (the slowest rank's time); the value
    itself when there is no process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(updates_per_rank, world, seconds):
    """Whole-job GLUPS of `world` replicas that each did updates_per_rank
    fluid updates, timed by the slowest rank."""
    return updates_per_rank * world / seconds / 1e9


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


def profiled_traffic(kernel_file, name, key="dram_bytes_per_launch_full_workload"):
    """DRAM bytes per launch (or per time step: key) from a committed ncu
    summary, if it was taken on the current kernel source (the summary
    records the source hash)."""
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
        return float(vals[key])
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


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(math.ceil(q / 100.0 * len(xs))) - 1))
    return xs[k]


def leg_precision(L, I, stream):
    """BF16 / FP16 shifted storage against the FP64 oracle on the 2048 x 1024
    tree: the first solve of the optimisation run (5000 steps from rest, same
    mask for all).  The oracle's solve is timed and doubles as the CPU
    baseline sample."""
    import numpy as np
    import oracle as ora
    cfg = I.config_tree_2048()
    cells, tau, u_max, S = cfg["cells"], cfg["tau"], cfg["u_max"], 5000
    ny, nx = cells.shape
    fluid = int((cells == 0).sum())
    s = ora.Solver(ora.make_params(nx, ny, tau, 1.0, u_max), cells, residual_every=0)
    t0 = time.perf_counter()
    o = s.solve(S)
    t_ora = time.perf_counter() - t0
    ref_frac = np.asarray(o["m_out"]) / np.sum(o["m_out"])
    out = {"workload": f"{cfg['name']} first solve, {S} steps from rest",
           "oracle": {"dp": o["dp"], "theta": o["theta"], "dg": o["dg"]}}
    glups = {}
    for name, pv in (("f32", L.F32), ("bf16", L.BF16_SHIFTED), ("f16", L.F16_SHIFTED)):
        h = L.Lattice(cells, tau, u_max, precision=pv, residual_every=0, stream=stream)
        r = h.solve(S)
        frac = np.asarray(r["m_out"]) / np.sum(r["m_out"])
        h.reset()
        h.kernel_time(reset=True)
        h.solve(S)
        ms, nl, nu = h.kernel_time()
        glups[name] = nu / (ms / 1e3) / 1e9
        out[name] = {"dp": r["dp"], "dp_rel_err": abs(r["dp"] - o["dp"]) / abs(o["dp"]),
                     "outlet_fraction_max_abs_err": float(np.max(np.abs(frac - ref_frac))),
                     "dg_abs_err": abs(r["dg"] - o["dg"]), "theta_abs_err": abs(r["theta"] - o["theta"]),
                     "glups_steps": glups[name], "glups_vs_f32": glups[name] / glups["f32"]}
        h.close()
    cores = ora.set_threads(0)
    # one host thread, on a short sample of the same lattice
    ora.set_threads(1)
    s1 = ora.Solver(ora.make_params(nx, ny, tau, 1.0, u_max), cells, residual_every=0)
    t0 = time.perf_counter()
    s1.solve(100)
    t_one = time.perf_counter() - t0
    ora.set_threads(cores)
    cpu = {"value": fluid * S / t_ora / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{cfg['name']}: the run's first solve, {S} FP64 time steps from rest, {t_ora:.1f} s",
           "single_thread_value": fluid * 100 / t_one / 1e9,
           "single_thread_sample": f"100 FP64 time steps of the same lattice on 1 thread, {t_one:.1f} s"}
    return out, cpu


def leg_tjunction(L, I, stream):
    """The 128 x 64 T-junction (1136 fluid cells, 10 x 2000 steps after a
    2000-step solve): on-chip and bound by the launch latency of a step."""
    c = I.config_t_junction()
    fluid = int((c["cells"] == 0).sum())
    h = L.Lattice(c["cells"], c["tau"], c["u_max"], residual_every=0, stream=stream)
    h.solve(256)
    h.reset()
    h.kernel_time(reset=True)
    t0 = time.perf_counter()
    out = h.optimize(2000, 10, 2)
    dt = time.perf_counter() - t0
    ms, nl, nu = h.kernel_time()
    res = {"fluid_cells": fluid, "glups": fluid * 2000 * 11 / dt / 1e9, "step_glups": nu / (ms / 1e3) / 1e9,
           "us_per_step": 1e3 * ms / nl, "dp_first": out["dp_first"], "dp_last": out["dp_last"],
           "step_config": list(h.step_config())}
    h.close()
    return res


def leg_collector(L, I, stream):
    """The paper's own LBM case, re-derived: the half-domain collector with a
    symmetry plane (Sec. 3.3), optimised from the first to the 151st step with
    lbm_optimize (5000 time steps per solve, n_swap = 0.2 % of the fluid)."""
    c = I.config_collector()
    fluid = int((c["cells"] == 0).sum())
    n_swap = max(1, fluid // 500)
    h = L.Lattice(c["cells"], c["tau"], c["u_max"], outlet=c["outlet"], residual_every=0, mirror=True,
                  stream=stream)
    h.solve(256)
    h.reset()
    h.kernel_time(reset=True)
    t0 = time.perf_counter()
    out = h.optimize(5000, c["n_iter"] - 1, n_swap)
    dt = time.perf_counter() - t0
    ms, nl, nu = h.kernel_time()
    first = out["history"][0]
    res = {"workload": f"{c['name']}: {c['n_iter']} solves of 5000 steps, n_swap {n_swap}, Re 22",
           "fluid_cells": fluid, "glups": fluid * 5000 * len(out["history"]) / dt / 1e9,
           "step_glups": nu / (ms / 1e3) / 1e9, "seconds": dt, "dp_first": first, "dp_last": out["dp_last"],
           "dp_best": out["dp_best"], "best_iter": out["best_iter"],
           "dp_change_first_to_best": out["dp_best"] / first - 1.0, "step_config": list(h.step_config())}
    h.close()
    return res


def leg_models(L, I, stream):
    """Cost of the collision models beyond BGK on the 2048 x 1024 tree (FP32):
    step GLUPS of a 5000-step solve with each model, and the oracle-free
    difference of the pressure drop to BGK (the models agree with BGK to
    first order at this Reynolds number)."""
    cfg = I.config_tree_2048()
    out = {}
    for name, coll, c in (("bgk", L.COLLIDE_BGK, 0.0), ("regularized", L.COLLIDE_REGULARIZED, 0.0),
                          ("smagorinsky_c0.1", L.COLLIDE_SMAGORINSKY, 0.1)):
        h = L.Lattice(cfg["cells"], cfg["tau"], cfg["u_max"], residual_every=0, collision=coll, c_smag=c,
                      stream=stream)
        h.solve(1000)
        h.reset()
        h.kernel_time(reset=True)
        r = h.solve(5000)
        ms, nl, nu = h.kernel_time()
        out[name] = {"glups_steps": nu / (ms / 1e3) / 1e9, "us_per_step": 1e3 * ms / nl, "dp": r["dp"],
                     "step_config": list(h.step_config())}
        h.close()
    for k in out:
        out[k]["glups_vs_bgk"] = out[k]["glups_steps"] / out["bgk"]["glups_steps"]
        out[k]["dp_rel_to_bgk"] = out[k]["dp"] / out["bgk"]["dp"] - 1.0
    return out


def oracle3_rate(cells, tau, u_max, seconds):
    """Fluid updates per second of the FP64 D3Q19 oracle on a bounded sample."""
    from oracle import lbm3d as o3
    nz, ny, nx = cells.shape
    p = o3.make_params3(nx, ny, nz, tau, u_max=u_max)
    u_in = o3.inlet_profile3(p, cells)
    f = o3.init3(p, cells)
    fluid = int((cells == 0).sum())
    n = 2
    while True:
        t0 = time.perf_counter()
        f, *_ = o3.run3(p, cells, u_in, f, n)
        t = time.perf_counter() - t0
        if t >= 0.25:
            break
        n *= 2
    n = max(2, int(seconds * n / t) // 2 * 2)
    t0 = time.perf_counter()
    o3.run3(p, cells, u_in, f, n)
    dt = time.perf_counter() - t0
    return fluid * n / dt, n, dt


def leg_d3q19(L, I, stream, peak, cpu_seconds=4.0):
    """The D3Q19 form of the path: step GLUPS and HBM fraction of the stream-
    collide kernels on the 384 x 192 x 192 distributor (FP32 and BF16
    storage) and on a full 256 x 128 x 128 duct, the optimisation loop on the
    distributor (exchange + re-solve), and the FP64 oracle's rate."""
    cfg = I.config_tree3d()
    out = {}
    cases = (("tree3d_384x192x192", cfg["cells"], cfg["tau"], cfg["u_max"]),
             ("duct3d_256x128x128", I.duct3d(256, 126, 126), 0.6, 0.05))
    for name, cells, tau, u_max in cases:
        fluid = int((cells == 0).sum())
        for pname, pv in (("f32", L.F32), ("bf16", L.BF16_SHIFTED)):
            h = L.Lattice3(cells, tau, u_max, precision=pv, stream=stream)
            h.solve(100)
            h.kernel_time(reset=True)
            r = h.solve(1000)
            ms, nl, nu = h.kernel_time()
            bpu = 2.0 * 19.0 * (4.0 if pv == L.F32 else 2.0) + 1.0 / 8.0
            gbs = fluid * bpu / ((ms / 1e3) / nl) / 1e9
            out[f"{name}_{pname}"] = {"fluid_cells": fluid, "glups": nu / (ms / 1e3) / 1e9,
                                      "us_per_step": 1e3 * ms / nl, "achieved_gbs": gbs,
                                      "frac_of_measured_hbm": gbs / peak, "dp": r["dp"]}
            h.close()
    for name, coll, c in (("regularized", L.COLLIDE_REGULARIZED, 0.0), ("smagorinsky_c0.1", L.COLLIDE_SMAGORINSKY, 0.1)):
        h = L.Lattice3(cfg["cells"], cfg["tau"], cfg["u_max"], collision=coll, c_smag=c, stream=stream)
        h.solve(100)
        h.kernel_time(reset=True)
        r = h.solve(1000)
        ms, nl, nu = h.kernel_time()
        out[f"tree3d_384x192x192_f32_{name}"] = {"glups": nu / (ms / 1e3) / 1e9, "us_per_step": 1e3 * ms / nl,
                                                 "glups_vs_bgk": (nu / (ms / 1e3) / 1e9)
                                                 / out["tree3d_384x192x192_f32"]["glups"],
                                                 "dp_rel_to_bgk": r["dp"] / out["tree3d_384x192x192_f32"]["dp"] - 1}
        h.close()
    h = L.Lattice3(cfg["cells"], cfg["tau"], cfg["u_max"], stream=stream)
    fluid = int((cfg["cells"] == 0).sum())
    n_swap = max(1, fluid // 500)
    t0 = time.perf_counter()
    first = h.solve(cfg["steps"])
    dps = [first["dp"]]
    for _ in range(5):
        dps.append(h.optimize_step(n_swap, cfg["steps"])["dp"])
    dt = time.perf_counter() - t0
    out["optimize_tree3d_f32"] = {"workload": f"{cfg['name']}: 6 solves of {cfg['steps']} steps, n_swap {n_swap}",
                                  "glups": fluid * cfg["steps"] * 6 / dt / 1e9, "seconds": dt, "dp": dps}
    h.close()
    # precision: 16-bit storage against the FP64 oracle on the 192 x 96 x 96 tree (800 steps from rest,
    # long enough for the flow to reach every outlet)
    import numpy as np
    from oracle import lbm3d as o3
    med = I.config_tree3d(192, 96, 96)
    nz, ny, nx = med["cells"].shape
    sv = o3.Solver3(o3.make_params3(nx, ny, nz, med["tau"], u_max=med["u_max"]), med["cells"])
    o = sv.solve(800)
    ref_frac = np.asarray(o["m_out"]) / np.sum(o["m_out"])
    prec = {"workload": f"{med['name']}, 800 steps from rest", "oracle_dp": o["dp"]}
    for pname, pv in (("f32", L.F32), ("bf16", L.BF16_SHIFTED), ("f16", L.F16_SHIFTED)):
        h = L.Lattice3(med["cells"], med["tau"], med["u_max"], precision=pv, stream=stream)
        r = h.solve(800)
        frac = np.asarray(r["m_out"]) / np.sum(r["m_out"])
        ux = h.read(L.FIELD3_UX).astype(np.float64)
        prec[pname] = {"dp_rel_err": abs(r["dp"] - o["dp"]) / abs(o["dp"]),
                       "outlet_fraction_max_abs_err": float(np.max(np.abs(frac - ref_frac))),
                       "ux_max_err_rel": float(np.abs(ux - sv.ux).max() / np.abs(sv.ux).max())}
        h.close()
    out["precision_tree3d_192x96x96"] = prec
    small = I.config_tree3d_small()
    r, n, dt = oracle3_rate(small["cells"], small["tau"], small["u_max"], cpu_seconds)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out["oracle3_cpu"] = {"glups": r / 1e9, "cores": cores,
                          "sample": f"{small['name']}: {n} FP64 time steps, {dt:.1f} s"}
    return out


def leg_batched(L, I, stream, prec, n=256, iters=10, S=2000, sample=32, peak=None):
    """256 uneven candidate distributors in one batch (one launch per stage
    for all) against the same candidates one at a time through their own
    handles (a sample of them, creation excluded)."""
    cands = I.config_candidates(n)
    members = [dict(cells=c["cells"], tau=c["tau"], u_max=c["u_max"]) for c in cands]
    fluid = [int((c["cells"] == 0).sum()) for c in cands]
    n_swap = [max(1, f // 500) for f in fluid]
    b = L.Batch(members, precision=prec, residual_every=0, stream=stream)
    b.solve(S)  # tunes the launch shape and captures the step graphs
    b.reset()
    b.kernel_time(reset=True)
    t0 = time.perf_counter()
    rb = b.solve(S)
    dp_b = [[x["dp"] for x in rb]]
    for _ in range(iters):
        rb = b.optimize_step(n_swap, S)
        dp_b.append([x["dp"] for x in rb])
    t_batch = time.perf_counter() - t0
    ms, nl, nu = b.kernel_time()
    w, g, pers, cpt, stg = b.step_config()
    n_groups = b.step_groups()
    b.close()
    upd = sum(fluid) * S * (iters + 1)
    idx = list(range(0, n, max(1, n // sample)))[:sample]
    t_plain, upd_plain, worst = 0.0, 0, 0.0
    for i in idx:
        c = cands[i]
        h = L.Lattice(c["cells"], c["tau"], c["u_max"], precision=prec, residual_every=0, stream=stream)
        h.solve(S)
        h.reset()
        t0 = time.perf_counter()
        r = h.solve(S)
        dps = [r["dp"]]
        for _ in range(iters):
            dps.append(h.optimize_step(n_swap[i], S)["dp"])
        t_plain += time.perf_counter() - t0
        h.close()
        upd_plain += fluid[i] * S * (iters + 1)
        for k, d in enumerate(dps):
            worst = max(worst, abs(d - dp_b[k][i]) / abs(d))
    g_batch = upd / t_batch / 1e9
    g_plain = upd_plain / t_plain / 1e9
    return {"candidates": n, "fluid_cells": sum(fluid), "iterations": iters, "steps_per_solve": S,
            "batched_glups": g_batch, "batched_step_glups": nu / (ms / 1e3) / 1e9,
            "batched_step_frac_of_measured_hbm": (nu / (ms / 1e3) * L.bytes_per_fluid_update(prec) / 1e9 / peak
                                                  if peak else None),
            "member_groups": n_groups,
            "batched_s": t_batch, "step_config": [w, g, pers, cpt, stg],
            "one_at_a_time_glups": g_plain, "one_at_a_time_sample": len(idx),
            "speedup": g_batch / g_plain, "dp_rel_diff_batched_vs_alone_max": worst}


def leg_served(L, I, prec, rate, seconds, seed=5, plain_sample=120):
    """Poisson request stream into the server (continuous batching), and the
    same requests served one at a time through handles (a sample, measured
    back to back with handle creation and tuning left out of the times; its
    queueing at the same arrivals is simulated from the measured service
    times)."""
    import threading
    arrivals = I.poisson_arrivals(rate, seconds, seed)

    def request(k):
        r = I.config_served_request(k)
        fl = int((r["cells"] == 0).sum())
        return r, fl, (max(1, fl // 500) if r["optimize"] else 0)

    srv = L.Server(precision=prec, max_active=1024, max_tick_steps=1000)
    for k in range(8):  # warm-up requests (graph capture, allocations)
        r, fl, ns = request(10_000_000 + k)
        srv.submit(-1 - k, r["cells"], r["tau"], r["u_max"], r["steps"], n_iter=min(r["n_iter"], 2), n_swap=ns)
    srv.wait_idle(120)
    srv.poll(64)
    base = srv.stats()
    meta = {}
    t_start = srv.now() + 0.05
    errors = []

    def submitter():
        try:
            for k, t in enumerate(arrivals):
                r, fl, ns = request(k)
                delay = t_start + t - srv.now()
                if delay > 0:
                    time.sleep(delay)
                meta[k] = (t_start + t, bool(r["optimize"]))
                srv.submit(k, r["cells"], r["tau"], r["u_max"], r["steps"], n_iter=r["n_iter"], n_swap=ns)
        except Exception as e:  # reported in the result
            errors.append(repr(e))

    th = threading.Thread(target=submitter)
    th.start()
    done = {}
    deadline = time.time() + 4 * seconds + 120
    while len(done) < len(arrivals) and time.time() < deadline:
        for d in srv.poll(1024, wait_ms=100):
            done[d["tag"]] = d
        if errors:
            break
    th.join()
    st = srv.stats()
    srv.close()
    lat = [done[k]["t_done"] - meta[k][0] for k in done if k in meta]
    lat_s = [done[k]["t_done"] - meta[k][0] for k in done if k in meta and not meta[k][1]]
    lat_o = [done[k]["t_done"] - meta[k][0] for k in done if k in meta and meta[k][1]]
    upd = sum(d["fluid_updates"] for d in done.values())
    t_end = max(d["t_done"] for d in done.values()) if done else t_start
    out = {"rate_hz": rate, "window_s": seconds, "requests": len(arrivals), "completed": len(done),
           "failed": sum(1 for d in done.values() if d["status"] != 0), "submit_errors": errors,
           "optimize_share": sum(1 for v in meta.values() if v[1]) / max(1, len(meta)),
           "p50_ms": 1e3 * pct(lat, 50), "p99_ms": 1e3 * pct(lat, 99),
           "p50_ms_solve": 1e3 * pct(lat_s, 50) if lat_s else None, "p99_ms_solve": 1e3 * pct(lat_s, 99) if lat_s else None,
           "p50_ms_optimize": 1e3 * pct(lat_o, 50) if lat_o else None,
           "p99_ms_optimize": 1e3 * pct(lat_o, 99) if lat_o else None,
           "aggregate_glups": upd / (t_end - t_start) / 1e9, "offered_glups": upd / seconds / 1e9,
           "gpu_step_glups": (st["fluid_updates"] - base["fluid_updates"]) /
                             max(1e-9, (st["step_ms"] - base["step_ms"]) / 1e3) / 1e9,
           "ticks": st["ticks"] - base["ticks"], "peak_active": st["peak_active"],
           "peak_resident_gb": st["peak_resident_bytes"] / 1e9, "peak_device_gb": st["peak_device_bytes"] / 1e9,
           "budget_gb": st["budget_bytes"] / 1e9, "scheduler_busy_s": st["busy_s"] - base["busy_s"]}
    if plain_sample <= 0:
        return out
    # one at a time through handles, back to back, on the first requests
    service, upd_p, worst = [], 0, 0.0
    for k in range(min(plain_sample, len(arrivals))):
        r, fl, ns = request(k)
        h = L.Lattice(r["cells"], r["tau"], r["u_max"], precision=prec, residual_every=0)
        h.solve(256)  # creation, launch-shape tuning and graph capture stay out of the timing
        h.reset()
        t0 = time.perf_counter()
        x = h.solve(r["steps"])
        for _ in range(r["n_iter"]):
            x = h.optimize_step(ns, r["steps"])
        service.append(time.perf_counter() - t0)
        h.close()
        upd_p += fl * r["steps"] * (1 + r["n_iter"])
        if k in done and done[k]["status"] == 0:
            worst = max(worst, abs(done[k]["last"]["dp"] - x["dp"]) / abs(x["dp"]))
    mean_service = sum(service) / len(service)
    # FIFO queue at the same arrival times with the measured service times (cycled)
    free_at, sim = 0.0, []
    for k, t in enumerate(arrivals):
        begin = max(t, free_at)
        free_at = begin + service[k % len(service)]
        sim.append(free_at - t)
    out["one_at_a_time"] = {"sample": len(service), "glups": upd_p / sum(service) / 1e9,
                            "mean_service_ms": 1e3 * mean_service, "utilisation_at_rate": rate * mean_service,
                            "simulated_p50_ms": 1e3 * pct(sim, 50), "simulated_p99_ms": 1e3 * pct(sim, 99),
                            "simulated_makespan_s": free_at}
    out["served_vs_alone_dp_rel_diff_max"] = worst
    out["speedup_aggregate"] = out["aggregate_glups"] / out["one_at_a_time"]["glups"]
    return out


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
    fluid = int((cfg["cells"] == 0).sum())
    S, iters, S0 = args.lattice_steps, args.iters, args.first_steps
    # the GPU arm's config (the same workload); the oracle times a bounded sample of it
    config = {"workload": cfg["name"] + f"_{args.precision}_{S0}+{iters}x{S}", "nx": cfg["nx"], "ny": cfg["ny"],
              "fluid_cells": fluid, "n_swap": max(1, int(0.002 * fluid)), "solves_per_step": iters + 1,
              "first_solve_steps": S0, "time_steps_per_solve": S, "l2": "flushed between timed steps (256 MB write)",
              "parallelism": f"replicas x{args.gpus}"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
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
    S, iters, S0 = args.lattice_steps, args.iters, args.first_steps
    stream = torch.cuda.Stream()
    lat = L.Lattice(cells, cfg["tau"], cfg["u_max"], precision=prec, residual_every=100, stream=stream)

    def one_run(handle):
        handle.reset()
        t0 = time.perf_counter()
        r = handle.solve(S0)
        r["wall_s"] = time.perf_counter() - t0
        hist = [r]
        for _ in range(iters):
            t0 = time.perf_counter()
            r = handle.optimize_step(n_swap, S)
            r["wall_s"] = time.perf_counter() - t0
            hist.append(r)
        return hist

    log = open(args.log, "w") if (args.log and rank == 0) else None

    def log_run(run, hist):
        if log is None:
            return
        for it, r in enumerate(hist):
            rec = {"run": run, "iteration": it, "steps": S0 if it == 0 else S, "dp": r["dp"], "m_in": r["m_in"],
                   "residual": r["residual"], "theta": r["theta"], "dg": r["dg"],
                   "m_out": [float(x) for x in r["m_out"]], "fluid_cells": r["fluid_cells"],
                   "n_swapped": r.get("n_swapped", 0), "steps_done": r["steps_done"], "wall_s": r["wall_s"]}
            log.write(json.dumps(rec) + "\n")

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
    runs = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)  # evict the lattice from L2 between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        last = one_run(lat)
        e1.record(stream)
        ev.append((e0, e1))
        runs.append(last)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = L.kernel_launches() - launches0
    for k, hist in enumerate(runs):  # after the timed region: the log costs it nothing
        log_run(k, hist)
    if log is not None:
        log.close()
    k_ms, k_launches, k_updates = lat.kernel_time()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    updates_per_step = fluid * (S0 + S * iters)
    total_s = max_over_ranks(total_s, dist, "cuda")
    value = replica_value(updates_per_step * args.steps, world, total_s)

    # roofline of the stream-collide kernel, from the timed region
    bpu = L.bytes_per_fluid_update(prec)
    avg_launch_s = (k_ms / 1e3) / max(k_launches, 1)
    bytes_per_launch = fluid * bpu
    achieved = bytes_per_launch / avg_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    resident = lat.step_config()[2] == 2
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (profiled_traffic("resident.cu", "resident_tree_2048x1024.md",
                                             "dram_bytes_per_step_full_workload") if resident
                            else profiled_traffic("step.cu", "stream_collide_tree_2048x1024.md")),
                "peak_kind": peak_kind, "bytes_per_launch": bytes_per_launch,
                "avg_launch_us": avg_launch_s * 1e6,
                "per": "time step (fluid cells x algorithmic bytes per update; mean time per step)",
                "kernel": "k_stream_collide_resident" if resident else "k_stream_collide",
                "note": ("populations in shared memory for the whole solve (one launch per solve), halo words in L2; "
                         "bound by SM instruction issue" if resident else
                         "lattice working set (fluid cells) is L2-resident within a solve")}

    # end to end through the public API, as many runs as timed steps: pinned
    # host cell map in, the whole optimisation run, the cell map back out.
    # The bytes crossing are the library's own count of its host <-> device
    # copies (uploads of the cell map and tables, result blocks, exchange
    # counters, the final read).
    cells_pin = torch.from_numpy(cells).pin_memory()
    mask_out = torch.empty(cells.shape, dtype=torch.uint8).pin_memory()
    e2e_times = []
    x0 = L.transfer_bytes()
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = L.Lattice(cells_pin.numpy(), cfg["tau"], cfg["u_max"], precision=prec, residual_every=100,
                      stream=stream)
        r = h.solve(S0)
        for _ in range(iters):
            r = h.optimize_step(n_swap, S)
        h.read(L.FIELD_MASK, out=mask_out.numpy())
        h.close()
        e2e_times.append(time.perf_counter() - t0)
    x1 = L.transfer_bytes()
    e2e_s = sum(e2e_times) / len(e2e_times)
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e = {"value": replica_value(updates_per_step, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": (x1[0] - x0[0]) // args.steps, "d2h_bytes_per_step": (x1[1] - x0[1]) // args.steps,
           "ms_per_step": 1e3 * e2e_s, "runs": args.steps,
           "bytes_source": "library transfer counters (lbm_transfer_bytes)"}

    extras = {}
    legs = set() if args.no_extras else set(x for x in args.legs.split(",") if x)
    cpu = None
    if rank == 0 and "large" in legs:
        # beyond-L2 lattice: 8192 x 4096 array of 16 straight channels (~50 % fluid)
        big = I.channel_array(8192, 4096, 16, fill=0.5)
        bf = int((big == 0).sum())
        for pname, pv in (("f32", L.F32), ("bf16", L.BF16_SHIFTED), ("f16", L.F16_SHIFTED)):
            hb = L.Lattice(big, 0.6, 0.05, precision=pv, residual_every=0, stream=stream)
            hb.solve(300)  # the first solve of 256 steps or more picks the launch shape
            hb.kernel_time(reset=True)
            hb.solve(400)
            ms, nl, nu = hb.kernel_time()
            gbs = bf * L.bytes_per_fluid_update(pv) / ((ms / 1e3) / nl) / 1e9
            extras[f"large_8192x4096_{pname}"] = {"glups": nu / (ms / 1e3) / 1e9, "achieved_gbs": gbs,
                                                  "frac_of_measured_hbm": gbs / peak, "fluid_cells": bf,
                                                  "step_config": list(hb.step_config()),
                                                  "windows": hb.task_counts()[1]}
            hb.close()
    if rank == 0 and "d3q19" in legs:
        extras["d3q19"] = leg_d3q19(L, I, stream, peak)
    if rank == 0 and "precision" in legs:
        extras["precision_tree_2048"], cpu_p = leg_precision(L, I, stream)
        if world == 1:
            cpu = cpu_p
    if rank == 0 and "tjunction" in legs:
        extras["t_junction_128x64"] = leg_tjunction(L, I, stream)
    if rank == 0 and "collector" in legs:
        extras["collector_half_360x180"] = leg_collector(L, I, stream)
    if rank == 0 and "models" in legs:
        extras["collision_models_tree_2048"] = leg_models(L, I, stream)
    if rank == 0 and "batched" in legs:
        for pname, pv in (("f32", L.F32), ("bf16", L.BF16_SHIFTED)):
            extras[f"batched_256_{pname}"] = leg_batched(L, I, stream, pv, peak=peak)
    if rank == 0 and "served" in legs:
        extras["served_f32"] = leg_served(L, I, L.F32, args.serve_rate, args.serve_seconds)
    if rank == 0 and "sweep" in legs:
        extras["served_sweep_f32"] = {str(int(r)): leg_served(L, I, L.F32, r, 10.0, plain_sample=0)
                                      for r in (50.0, 100.0, 200.0, 400.0)}
    if cpu is None and legs and rank == 0 and world == 1:
        r, n, dt, cores = oracle_rate(cells, cfg["tau"], cfg["u_max"], args.cpu_seconds)
        cpu = {"value": r / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{cfg['name']}: {n} FP64 time steps from rest, {dt:.1f} s"}

    if rank == 0:
        dp_hist = [r["dp"] for r in last]
        r_last = last[-1]
        best_iter = min(range(len(dp_hist)), key=lambda k: dp_hist[k])
        summary = {"summary": "per-leg rates (the full records are in the main line's extras)",
                   "headline_glups": value, "headline_roofline_frac": roofline["frac"],
                   "e2e_glups": e2e["value"]}
        summary.update(leg_summary(extras))
        print(json.dumps(summary))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == L.F32 else args.precision,
                "data": "synthetic",
                "config": {"workload": cfg["name"] + f"_{args.precision}_{S0}+{iters}x{S}", "nx": cfg["nx"],
                           "ny": cfg["ny"], "fluid_cells": fluid, "n_swap": n_swap,
                           "solves_per_step": iters + 1, "first_solve_steps": S0, "time_steps_per_solve": S,
                           "l2": "flushed between timed steps (256 MB write)",
                           "parallelism": f"replicas x{world}"},
                "step_config": dict(zip(("warps_per_block", "grid", "persistent", "cells_per_thread", "stages"),
                                        lat.step_config())),
                "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
                "cpu_baseline": cpu,
                "dense_glups": cfg["nx"] * cfg["ny"] * (S0 + S * iters) * args.steps * world / total_s / 1e9,
                "dp_initial": dp_hist[0], "dp_best": dp_hist[best_iter], "best_iter": best_iter,
                "dp_final": r_last["dp"], "theta_initial": last[0]["theta"], "theta_final": r_last["theta"],
                "dg_initial": last[0]["dg"], "dg_final": r_last["dg"],
                "dp_history": dp_hist, "theta_history": [r["theta"] for r in last], "extras": extras}
        print(json.dumps(line))
    lat.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def leg_summary(extras):
    """Compact rates of every leg that ran, for a short line ahead of the main one."""
    out = {}

    def put(key, d, field):
        if isinstance(d, dict) and d.get(field) is not None:
            out[key] = d[field]

    for p in ("f32", "bf16", "f16"):
        put(f"large_{p}_glups", extras.get(f"large_8192x4096_{p}"), "glups")
        put(f"large_{p}_frac", extras.get(f"large_8192x4096_{p}"), "frac_of_measured_hbm")
    for p in ("f32", "bf16"):
        put(f"batched_{p}_glups", extras.get(f"batched_256_{p}"), "batched_glups")
        put(f"batched_{p}_step_glups", extras.get(f"batched_256_{p}"), "batched_step_glups")
        put(f"batched_{p}_speedup", extras.get(f"batched_256_{p}"), "speedup")
        put(f"batched_{p}_step_frac", extras.get(f"batched_256_{p}"), "batched_step_frac_of_measured_hbm")
    prec = extras.get("precision_tree_2048", {})
    for p in ("bf16", "f16"):
        put(f"tree_{p}_vs_f32", prec.get(p), "glups_vs_f32")
        put(f"tree_{p}_dp_rel_err", prec.get(p), "dp_rel_err")
    d3 = extras.get("d3q19", {})
    for k in ("tree3d_384x192x192_f32", "tree3d_384x192x192_bf16", "duct3d_256x128x128_f32"):
        put(f"{k}_glups", d3.get(k), "glups")
        put(f"{k}_frac", d3.get(k), "frac_of_measured_hbm")
    srv = extras.get("served_f32", {})
    for k in ("p50_ms", "p99_ms", "aggregate_glups", "served_vs_alone_dp_rel_diff_max"):
        put(f"served_{k}", srv, k)
    put("tjunction_glups", extras.get("t_junction_128x64"), "glups")
    put("collector_glups", extras.get("collector_half_360x180"), "glups")
    return out


if __name__ == "__main__":
    sys.exit(main())
