"""Strip decomposition of one lattice over two CPU ranks (gloo): the halo
exchange of the populations crossing each cut reproduces the single-domain
oracle bit for bit, including the reductions done on rank 0.  A rank that
fails between steps is reported to the launcher, not hung."""
import multiprocessing as mp
import socket

import numpy as np

from paper_1303_0107_gb300 import inputs as I


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _launch(world, args, fail_rank=-1, timeout=120):
    import _decomp_worker
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_decomp_worker.worker, args=(r, world, port, *args, fail_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout)
    codes = []
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
        codes.append(p.exitcode)
    return codes


def test_two_rank_strips_equal_single_domain(ora, tmp_path):
    cfg = I.config_t_junction()
    nx, ny, steps = cfg["nx"], cfg["ny"], 60
    out = str(tmp_path / "decomp.npz")
    codes = _launch(2, (nx, ny, steps, cfg["cells"], cfg["u_max"], cfg["tau"], out))
    assert codes == [0, 0]
    got = np.load(out)
    p = ora.make_params(nx, ny, cfg["tau"], 1.0, cfg["u_max"])
    u_in = ora.inlet_profile(p, cfg["cells"])
    f, rho, ux, uy, st = ora.run(p, cfg["cells"], u_in, ora.init(p, cfg["cells"]), steps)
    assert np.array_equal(got["f"], f)
    assert np.array_equal(got["rho"], rho) and np.array_equal(got["ux"], ux)
    dp_a = ora.observables(p, cfg["cells"], got["rho"], got["ux"])
    dp_b = ora.observables(p, cfg["cells"], rho, ux)
    assert dp_a[0] == dp_b[0] and np.array_equal(dp_a[2], dp_b[2])


def test_failed_rank_is_reported(tmp_path):
    cfg = I.config_t_junction()
    out = str(tmp_path / "never.npz")
    codes = _launch(2, (cfg["nx"], cfg["ny"], 20, cfg["cells"], cfg["u_max"], cfg["tau"], out),
                    fail_rank=1, timeout=60)
    assert codes[1] != 0
    assert codes[0] != 0  # rank 0 sees the peer's exit as an error, it does not hang
