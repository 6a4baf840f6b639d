"""Seeded synthetic inputs: cell-type maps of distributor trees and test domains.

This module only draws geometry (integer cell maps) and workload recipes; it
holds none of the lattice Boltzmann arithmetic, so both the CUDA path and the
CPU oracle can be fed from it.  Cell maps are uint8 arrays of shape (ny, nx),
row-major, 1 = solid, 0 = fluid; x runs along the flow, y across.

The paper's own geometry figures are not available, so the distributor is
drawn from its description (Sec. 3.2): a binary tree of T-bifurcations fed by
one inlet channel, 2^G parallel outlets, segment lengths in the 2:2:1:1
proportion of Eq. 7 (the inlet trunk counted as 2), widths shrinking by a
ratio r per generation.
"""
import json
import math
import os

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed: int, counter: int) -> int:
    """SplitMix64 output for state seed + (counter+1)*golden (Steele, Lea & Flood 2014)."""
    z = (seed + (counter + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def uniform01(seed: int, counter: int) -> float:
    return (splitmix64(seed, counter) >> 11) * (1.0 / (1 << 53))


def _fill(cells, x0, x1, y0, y1):
    ny, nx = cells.shape
    cells[max(y0, 1):min(y1, ny - 1), max(x0, 0):min(x1, nx)] = 0


def tree_widths(w0: int, ratio: float, generations: int, min_width: int = 3):
    return [max(min_width, int(round(w0 * ratio ** k))) for k in range(generations + 1)]


def tree(nx: int, ny: int, generations: int, w0: int, ratio: float = 0.5, jitter: int = 2,
         seed: int = 0, widths=None, lengths=(2, 2, 2, 1, 1)) -> np.ndarray:
    """Arborescent distributor: one inlet on x = 0, 2^G outlets on x = nx-1.

    Generation 0 is the trunk of width W0 centred on y = ny/2.  A node of
    generation k (k = 1..G) sits at x = X_k (+ jitter) and is a vertical bar of
    width W_k spanning its parent's centre +- s_k, s_k = ny / 2^(k+1); two
    horizontal children of width W_k leave the bar ends towards the next
    generation (or the outlet column for k = G).  X_k follows the segment
    lengths `lengths` (Eq. 7 proportions), unit = nx / sum(lengths[:G+1]).
    Each node is shifted by an integer in [-jitter, jitter] drawn from
    splitmix64(seed, node id), node id = 2^(k-1) + j in heap order.
    """
    G = int(generations)
    if widths is None:
        widths = tree_widths(w0, ratio, G)
    widths = [int(w) for w in widths]
    lens = list(lengths[:G + 1])
    unit = nx / float(sum(lens))
    xs_nominal = [int(round(unit * sum(lens[:k]))) for k in range(G + 1)]  # X_0 = 0 .. X_G
    cells = np.ones((ny, nx), np.uint8)

    def node_x(k, j):
        if jitter <= 0:
            return xs_nominal[k]
        node_id = (1 << (k - 1)) + j
        shift = int(splitmix64(seed, node_id) % (2 * jitter + 1)) - jitter
        return xs_nominal[k] + shift

    def hchannel(yc, w, x0, x1):
        _fill(cells, x0, x1, yc - w // 2, yc - w // 2 + w)

    yc0 = ny // 2
    if G == 0:
        hchannel(yc0, widths[0], 0, nx)
        return cells
    # trunk: from the inlet to the far side of the first bar
    x1 = node_x(1, 0)
    hchannel(yc0, widths[0], 0, x1 + widths[1])
    # level by level: (centre y, x of the node) of every node of generation k
    level = [(yc0, x1)]
    for k in range(1, G + 1):
        s = ny >> (k + 1)
        wk = widths[k]
        nxt = []
        for j, (yc, xk) in enumerate(level):
            # vertical bar of the T
            _fill(cells, xk, xk + wk, yc - s - wk // 2, yc + s - wk // 2 + wk)
            for side, yc_child in enumerate((yc - s, yc + s)):
                if k < G:
                    jj = 2 * j + side
                    x_next = node_x(k + 1, jj)
                    hchannel(yc_child, wk, xk, x_next + widths[k + 1])
                    nxt.append((yc_child, x_next))
                else:
                    hchannel(yc_child, wk, xk, nx)
        level = nxt
    return cells


def channel(nx: int, height: int) -> np.ndarray:
    """Straight channel of `height` fluid rows between two walls, open at both ends."""
    cells = np.ones((height + 2, nx), np.uint8)
    cells[1:height + 1, :] = 0
    return cells


def box(nx: int, ny: int) -> np.ndarray:
    """Closed box: fluid inside a one-cell solid frame on all four sides."""
    cells = np.ones((ny, nx), np.uint8)
    cells[1:ny - 1, 1:nx - 1] = 0
    return cells


def channel_array(nx: int, ny: int, n_channels: int, fill: float = 0.5) -> np.ndarray:
    """n straight parallel channels across the whole length (fluid fraction ~fill)."""
    cells = np.ones((ny, nx), np.uint8)
    pitch = ny // n_channels
    h = max(1, int(round(pitch * fill)))
    for c in range(n_channels):
        y0 = c * pitch + (pitch - h) // 2
        _fill(cells, 0, nx, y0, y0 + h)
    return cells


def random_blobs(nx: int, ny: int, seed: int, density: float = 0.15) -> np.ndarray:
    """Channel with random solid obstacles (interior only), for parity of irregular walls."""
    cells = channel(nx, ny - 2)
    for y in range(1, ny - 1):
        for x in range(3, nx - 3):
            if uniform01(seed, y * nx + x) < density:
                cells[y, x] = 1
    return cells


# ---------------------------------------------------------------------------
# Three-dimensional cell maps: uint8 arrays of shape (nz, ny, nx), 1 = solid.
# ---------------------------------------------------------------------------

def extrude(cells2d: np.ndarray, depth: int) -> np.ndarray:
    """A plate device of finite depth: the 2D map repeated over `depth` fluid
    layers z = 1..depth between two solid plates (z = 0 and z = depth + 1)."""
    ny, nx = cells2d.shape
    out = np.ones((depth + 2, ny, nx), np.uint8)
    out[1:depth + 1] = cells2d[None]
    return out


def tree3d(nx: int, ny: int, nz: int, generations: int, w0: int, ratio: float = 2.0 ** (-1.0 / 3.0),
           min_width: int = 3) -> np.ndarray:
    """Binary distributor of square ducts: a trunk of width w0 on the axis
    (ny/2, nz/2) from x = 0 splits 2^G ways, generation k (k = 0, 1, ...)
    splitting along y when k is even and along z when k is odd, each child
    taking the middle of its half of the parent's cross-section.  A split is
    a header duct across the split axis at the parent's last w_k columns.
    Widths w_k = max(min_width, round(w0 ratio^k)) (ratio 2^(-1/3): Murray's
    law for equal children); the trunk is two segments long, every
    generation one, segment = nx // (G + 2); the last generation runs out to
    x = nx - 1, giving 2^G outlet regions."""
    cells = np.ones((nz, ny, nx), np.uint8)
    seg = nx // (generations + 2)
    widths = [max(min_width, int(round(w0 * ratio ** k))) for k in range(generations + 1)]

    def carve(z0, z1, y0, y1, x0, x1):
        cells[max(z0, 1):min(z1, nz - 1), max(y0, 1):min(y1, ny - 1), max(x0, 0):min(x1, nx)] = 0

    def rec(k, x0, yc, zc, hy, hz):
        w = widths[k]
        x1 = nx if k == generations else x0 + (2 * seg if k == 0 else seg)
        carve(zc - w // 2, zc - w // 2 + w, yc - w // 2, yc - w // 2 + w, x0, x1)
        if k == generations:
            return
        wc = widths[k + 1]
        if k % 2 == 0:
            c1, c2 = yc - hy // 2, yc + hy // 2
            carve(zc - w // 2, zc - w // 2 + w, c1 - wc // 2, c2 - wc // 2 + wc, x1 - w, x1)
            rec(k + 1, x1 - wc, c1, zc, hy // 2, hz)
            rec(k + 1, x1 - wc, c2, zc, hy // 2, hz)
        else:
            c1, c2 = zc - hz // 2, zc + hz // 2
            carve(c1 - wc // 2, c2 - wc // 2 + wc, yc - w // 2, yc - w // 2 + w, x1 - w, x1)
            rec(k + 1, x1 - wc, yc, c1, hy, hz // 2)
            rec(k + 1, x1 - wc, yc, c2, hy, hz // 2)

    rec(0, 0, ny // 2, nz // 2, ny // 2, nz // 2)
    return cells


def duct3d(nx: int, wy: int, wz: int) -> np.ndarray:
    """Straight rectangular duct of wy x wz fluid cells, open at both ends."""
    cells = np.ones((wz + 2, wy + 2, nx), np.uint8)
    cells[1:wz + 1, 1:wy + 1, :] = 0
    return cells


def random_blobs3d(nx: int, ny: int, nz: int, seed: int, density: float = 0.15) -> np.ndarray:
    """Duct with random solid cells (x in [3, nx-4]), for parity of irregular walls."""
    cells = duct3d(nx, ny - 2, nz - 2)
    for z in range(1, nz - 1):
        for y in range(1, ny - 1):
            for x in range(3, nx - 3):
                if uniform01(seed, (z * ny + y) * nx + x) < density:
                    cells[z, y, x] = 1
    return cells


# ---------------------------------------------------------------------------
# Workload recipes.  Lattice units: dx = dt = 1, rho0 = 1.  The five
# benchmark workloads are described by the JSON files in configs/ (the
# generator and its parameters, tau, u_max, steps, iterations); the
# functions below build them from those files.
# ---------------------------------------------------------------------------

CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")
CONFIG_NAMES = ("t_junction_128x64", "tree_2048x1024_g4", "tree_2048x1024_g4_16bit", "candidates_256",
                "served_poisson_200")


def load_config(name: str) -> dict:
    """The recipe configs/<name>.json (one of CONFIG_NAMES) as a dict."""
    with open(os.path.join(CONFIG_DIR, name + ".json")) as f:
        return json.load(f)


def _tree_from(geo: dict, seed=None):
    return tree(geo["nx"], geo["ny"], geo["generations"], geo["w0"], widths=geo.get("widths"),
                jitter=geo["jitter"], seed=geo["seed"] if seed is None else seed)


def config_t_junction(seed: int = 0):
    """128 x 64, one T: inlet 8 wide, two outlets 4 wide; tau 0.8, u_max 0.05, 10 x 2000 steps."""
    c = load_config("t_junction_128x64")
    g = c["geometry"]
    return dict(name=c["name"], cells=_tree_from(g, seed), nx=g["nx"], ny=g["ny"], tau=c["tau"],
                u_max=c["u_max"], n_iter=c["n_iter"], steps=c["steps"])


def config_tree_2048(seed: int = 0):
    """2048 x 1024, four generations, widths 64/32/16/8/4, jitter +-2; Re = 50 on the
    64-wide inlet at nu = 0.01 (tau 0.53): mean inlet speed 0.0078125, u_max = 1.5x that."""
    c = load_config("tree_2048x1024_g4")
    g = c["geometry"]
    return dict(name=c["name"], cells=_tree_from(g, seed), nx=g["nx"], ny=g["ny"], tau=c["tau"],
                u_max=c["u_max"], n_iter=c["n_iter"], steps=c["steps"], first_solve_steps=c["first_solve_steps"],
                n_swap=c["n_swap"])


def config_collector():
    """The paper's own LBM case, re-derived (Sec. 3.3; its figures are not
    available): an arborescent collector on a half domain of 360 x 180 cells
    (flow along x) with a symmetry plane below row 0.  Eight inlets of 11
    cells on column 0 (sixteen in the whole domain), one outlet of 52 cells
    on column 359 against the plane (104 in the whole domain), joined by a
    four-generation binary tree with Eq. 7's 2:2:1:1 segment lengths and
    widths shrinking by (11/104)^(1/4) per generation; parabolic inlets,
    rho0 = 1, and the paper's inlet Reynolds number Re = W_in u_in / nu = 22.
    The paper's lattice values (nu = 0.04, mean inlet speed 0.08) diverge on
    this geometry in both the oracle and the GPU path (density swings of a
    third within 2000 steps), so the same Re is taken at nu = 0.01
    (tau = 0.53) and a mean inlet speed of 0.02 (u_max 0.03).  The paper's
    zero-gradient outlet leaves the density level free: over the 151
    optimisation steps it climbs by an order of one (measured), so the
    outlet holds rho0 instead."""
    nx, ny_full = 360, 360
    ratio = (11.0 / 104.0) ** 0.25
    full = tree(nx, ny_full, 4, 104, ratio=ratio, jitter=0, seed=0)
    collector = full[:, ::-1]            # branches on column 0, trunk on column nx-1
    half = np.ascontiguousarray(collector[ny_full // 2:, :])  # rows above the plane
    return dict(name="collector_360x180_half", cells=half, nx=nx, ny=ny_full // 2, tau=0.53, u_max=0.03,
                outlet=0, mirror=True, n_iter=151)


def config_candidates(n: int = 256, base_seed: int = 0):
    """Uneven candidate distributors: nx log-uniform in [256, 1024] (multiple of 32),
    ny = nx/2, G in {2,3,4}, width ratio in [0.6, 0.8], W0 = ny/16; tau 0.53 and
    Re = 50 on the inlet (u_max = 1.5 * 50 * 0.01 / W0)."""
    c = load_config("candidates_256")
    lo, hi = c["nx_range"]
    mult = c["nx_multiple"]
    gens = c["generations"]
    out = []
    for k in range(n):
        s = base_seed + k
        u = uniform01(s, 1)
        nx = int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))) / float(mult))) * mult
        ny = nx // 2
        G = gens[0] + int(splitmix64(s, 2) % len(gens))
        r = c["ratio_min"] + c["ratio_span"] * uniform01(s, 3)
        w0 = max(c["w0_min"], ny // c["w0_divisor"])
        cells = tree(nx, ny, G, w0, ratio=r, jitter=c["jitter"], seed=s)
        out.append(dict(name=f"cand{k}", cells=cells, nx=nx, ny=ny, tau=c["tau"],
                        u_max=1.5 * c["reynolds"] * c["nu"] / w0, generations=G, ratio=r, seed=s))
    return out


def config_tree3d_small():
    """72 x 34 x 34 D3Q19 distributor, two generations (4 outlets), trunk 10 wide;
    tau 0.8, u_max 0.05."""
    cells = tree3d(72, 34, 34, 2, 10)
    return dict(name="tree3d_72x34x34_g2", cells=cells, nx=72, ny=34, nz=34, tau=0.8, u_max=0.05)


def config_tree3d(nx: int = 384, ny: int = 192, nz: int = 192):
    """D3Q19 distributor of 384 x 192 x 192 cells: four generations (16 outlet
    ducts), trunk 48 wide, widths shrinking by 2^(-1/3); Re = 50 on the trunk at
    nu = 0.01 (tau 0.53): mean inlet speed 50 * 0.01 / 48; the product of two
    parabolas has a mean of 4/9 of its peak, so u_max = 9/4 of the mean."""
    cells = tree3d(nx, ny, nz, 4, 48)
    return dict(name=f"tree3d_{nx}x{ny}x{nz}_g4", cells=cells, nx=nx, ny=ny, nz=nz, tau=0.53,
                u_max=2.25 * 50 * 0.01 / 48, steps=2000)


def config_served_request(seed: int):
    """One served request: nx log-uniform in [128, 2048], ny = nx/2,
    G = clamp(floor(log2(nx/128)) + 1, 1, 4), W0 = max(8, ny/16), r = 0.5."""
    c = load_config("served_poisson_200")
    lo, hi = c["nx_range"]
    mult = c["nx_multiple"]
    u = uniform01(seed, 11)
    nx = int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))) / float(mult))) * mult
    ny = nx // 2
    G = min(4, max(1, int(math.floor(math.log2(nx / float(lo)))) + 1))
    w0 = max(c["w0_min"], ny // c["w0_divisor"])
    cells = tree(nx, ny, G, w0, ratio=c["ratio"], jitter=c["jitter"], seed=seed)
    optimize = uniform01(seed, 12) < c["optimize_fraction"]
    return dict(name=f"req{seed}", cells=cells, nx=nx, ny=ny, tau=c["tau"],
                u_max=min(c["u_max_cap"], 1.5 * c["reynolds"] * c["nu"] / w0), optimize=optimize,
                steps=c["solve_steps"], n_iter=c["optimize_iterations"] if optimize else 0, seed=seed)


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int):
    """Arrival times (s) of a Poisson process: exponential gaps from splitmix64 uniforms."""
    t, k, out = 0.0, 0, []
    while True:
        u = uniform01(seed, 1000003 + k)
        t += -math.log(1.0 - u) / rate_hz
        if t >= duration_s:
            return out
        out.append(t)
        k += 1
