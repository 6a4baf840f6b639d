"""The five benchmark workloads as recipes in paper_1303_0107_gb300/configs/*.json: each file loads,
carries its documented keys, and the builders in inputs.py produce the lattices the recipes describe
(sizes, parameters, the tree's exchange size as 0.2 % of its fluid cells)."""
import json
import os

import numpy as np
import pytest

from paper_1303_0107_gb300 import inputs as I


def test_every_config_file_loads():
    names = sorted(f[:-5] for f in os.listdir(I.CONFIG_DIR) if f.endswith(".json"))
    assert names == sorted(I.CONFIG_NAMES)
    for n in names:
        c = I.load_config(n)
        assert c["name"] == n and c["description"]
        with open(os.path.join(I.CONFIG_DIR, n + ".json")) as f:
            assert json.load(f) == c


def test_t_junction_recipe():
    c = I.load_config("t_junction_128x64")
    t = I.config_t_junction()
    assert t["cells"].shape == (64, 128)
    assert (t["tau"], t["u_max"], t["n_iter"], t["steps"]) == (c["tau"], c["u_max"], c["n_iter"], c["steps"])
    assert (t["cells"][1:-1, 0] == 0).sum() == 8  # inlet 8 wide
    assert (t["cells"][1:-1, -1] == 0).sum() == 8  # two outlets 4 wide


def test_tree_recipe():
    c = I.load_config("tree_2048x1024_g4")
    t = I.config_tree_2048()
    assert t["cells"].shape == (1024, 2048)
    fluid = int((t["cells"] == 0).sum())
    assert c["n_swap"] == max(1, int(0.002 * fluid))
    assert (t["cells"][1:-1, 0] == 0).sum() == 64
    outlet = (t["cells"][1:-1, -1] == 0).astype(int)
    assert int((np.diff(outlet) == 1).sum()) == 16  # 16 outlet channels
    p = I.load_config("tree_2048x1024_g4_16bit")
    assert p["base"] == c["name"] and p["storage"] == ["bf16", "f16"]


def test_candidates_recipe():
    c = I.load_config("candidates_256")
    cands = I.config_candidates(c["n"])
    assert len(cands) == 256
    for k in cands:
        assert c["nx_range"][0] <= k["nx"] <= c["nx_range"][1] and k["nx"] % c["nx_multiple"] == 0
        assert k["cells"].shape == (k["nx"] // 2, k["nx"])
        assert k["generations"] in c["generations"]
        assert c["ratio_min"] <= k["ratio"] <= c["ratio_min"] + c["ratio_span"]
    assert len({k["nx"] for k in cands}) > 10  # uneven sizes


def test_served_recipe():
    c = I.load_config("served_poisson_200")
    reqs = [I.config_served_request(s) for s in range(200)]
    for r in reqs:
        assert c["nx_range"][0] <= r["nx"] <= c["nx_range"][1]
        assert r["steps"] == c["solve_steps"] and r["n_iter"] in (0, c["optimize_iterations"])
        assert r["u_max"] <= c["u_max_cap"]
    frac = np.mean([r["optimize"] for r in reqs])
    assert abs(frac - c["optimize_fraction"]) < 0.1
