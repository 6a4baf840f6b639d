"""The multi-GPU path of bench.py is replicas (one lattice per rank, no
collective on the data path): the only cross-rank step is taking the slowest
rank's time.  Checked here on two CPU ranks over gloo."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")  # rank 1 is the slow one
    v = bench.replica_value(3e9, world, t)
    dist.destroy_process_group()
    with open(f"{out}.{rank}", "w") as f:
        f.write(f"{t} {v}")


def test_slowest_rank_sets_the_time(tmp_path):
    ctx = mp.get_context("spawn")
    port = _free_port()
    out = str(tmp_path / "r")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
    assert [p.exitcode for p in procs] == [0, 0]
    for r in range(2):
        t, v = map(float, open(f"{out}.{r}").read().split())
        assert t == 2.5  # both ranks see the slower time
        assert abs(v - 3e9 * 2 / 2.5 / 1e9) < 1e-12


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.75, None, "cpu") == 0.75
    assert bench.replica_value(1e9, 1, 0.5) == 2.0


def test_reference_arm_other_ranks_exit_without_work():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, cpu_seconds, gpus = 1, 0, 0.1, 2
    assert bench.run_reference(A(), 2, 1) == 0


def test_leg_summary_picks_each_legs_rates():
    sys.path.insert(0, ROOT)
    import bench
    extras = {"large_8192x4096_f32": {"glups": 69.3, "frac_of_measured_hbm": 0.74, "fluid_cells": 1},
              "large_8192x4096_bf16": {"glups": 76.9, "frac_of_measured_hbm": 0.41},
              "batched_256_f32": {"batched_glups": 43.3, "batched_step_glups": 45.0, "speedup": 3.0},
              "precision_tree_2048": {"bf16": {"glups_vs_f32": 0.79, "dp_rel_err": 9.8e-3}},
              "d3q19": {"tree3d_384x192x192_f32": {"glups": 28.4, "frac_of_measured_hbm": 0.64}},
              "served_f32": {"p50_ms": 7.1, "p99_ms": 164.6, "aggregate_glups": 29.1}}
    s = bench.leg_summary(extras)
    assert s["large_f32_glups"] == 69.3 and s["large_bf16_frac"] == 0.41
    assert s["batched_f32_glups"] == 43.3 and s["batched_f32_speedup"] == 3.0
    assert s["tree_bf16_vs_f32"] == 0.79 and s["tree3d_384x192x192_f32_frac"] == 0.64
    assert s["served_p50_ms"] == 7.1 and s["served_aggregate_glups"] == 29.1
    assert "batched_bf16_glups" not in s  # legs that did not run are left out
    assert bench.leg_summary({}) == {}
