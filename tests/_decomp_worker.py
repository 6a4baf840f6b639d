"""Worker for the two-rank strip decomposition check (CPU, gloo).

Each rank owns a block of columns of one lattice; after every step it sends
its edge column of the new post-collision state to the neighbouring rank and
receives that rank's edge column (the populations crossing the cut).  The
per-cell update is the oracle's, so the decomposed run must give the same
bits as the single-domain run.
"""
import os

import numpy as np


def worker(rank, world, port, nx, ny, steps, cells, u_max, tau, result_path, fail_rank=-1):
    import torch
    import torch.distributed as dist
    import oracle as ora

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = ora.make_params(nx, ny, tau, 1.0, u_max)
        u_in = ora.inlet_profile(p, cells)
        f = ora.init(p, cells)
        cuts = [nx * r // world for r in range(world + 1)]
        x0, x1 = cuts[rank], cuts[rank + 1]
        fields = None
        for t in range(steps):
            if rank == fail_rank and t == steps // 2:
                raise RuntimeError("injected host-side failure")
            f_next, fields = ora.step_columns(p, cells, u_in, f, x0, x1)
            # exchange the edge columns of the new state with the neighbours
            reqs = []
            if rank > 0:
                send_l = torch.from_numpy(np.ascontiguousarray(f_next[:, :, x0]))
                recv_l = torch.empty_like(send_l)
                reqs += [dist.isend(send_l, rank - 1), dist.irecv(recv_l, rank - 1)]
            if rank < world - 1:
                send_r = torch.from_numpy(np.ascontiguousarray(f_next[:, :, x1 - 1]))
                recv_r = torch.empty_like(send_r)
                reqs += [dist.isend(send_r, rank + 1), dist.irecv(recv_r, rank + 1)]
            for r in reqs:
                r.wait()
            if rank > 0:
                f_next[:, :, x0 - 1] = recv_l.numpy()
            if rank < world - 1:
                f_next[:, :, x1] = recv_r.numpy()
            f = f_next
        # gather owned columns on rank 0
        own = torch.from_numpy(np.ascontiguousarray(np.concatenate(
            [f[:, :, x0:x1].reshape(-1), np.stack(fields)[:, :, x0:x1].reshape(-1)])))
        sizes = [(cuts[r + 1] - cuts[r]) * ny * 12 for r in range(world)]
        if rank == 0:
            bufs = [torch.empty(s, dtype=torch.float64) for s in sizes]
            bufs[0].copy_(own)
            for r in range(1, world):
                dist.recv(bufs[r], r)
            f_all = np.zeros((9, ny, nx))
            fl_all = np.zeros((3, ny, nx))
            for r in range(world):
                w = cuts[r + 1] - cuts[r]
                b = bufs[r].numpy()
                f_all[:, :, cuts[r]:cuts[r + 1]] = b[:9 * ny * w].reshape(9, ny, w)
                fl_all[:, :, cuts[r]:cuts[r + 1]] = b[9 * ny * w:].reshape(3, ny, w)
            np.savez(result_path, f=f_all, rho=fl_all[0], ux=fl_all[1], uy=fl_all[2])
        else:
            dist.send(own, 0)
    finally:
        dist.destroy_process_group()
