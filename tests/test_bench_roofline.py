"""bench.py's roofline entry takes its DRAM traffic from a committed ncu
summary only while that summary was taken on the current kernel source (the
summary records the source hash); otherwise the traffic is null.  Checked
on the committed files and on a copy with the hash changed (CPU only)."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_committed_tree_summary_is_read_only_for_its_source():
    src = os.path.join(ROOT, "paper_1303_0107_gb300", "csrc", "step.cu")
    summ = os.path.join(ROOT, "profiles", "stream_collide_tree_2048x1024.md")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    t = bench.profiled_traffic("step.cu", "stream_collide_tree_2048x1024.md")
    if f"source_sha256_16: {h}" in open(summ).read():
        assert t is not None and 8e6 < t < 1.2e7  # bytes per launch of the benchmark lattice
    else:  # the kernel changed since the capture: no traffic claimed
        assert t is None


def test_traffic_is_null_once_the_source_hash_differs(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1303_0107_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("// kernel v1\n")
    h1 = hashlib.sha256(b"// kernel v1\n").hexdigest()[:16]
    (tmp_path / "profiles" / "k.md").write_text(
        f"source_sha256_16: {h1}\ndram_bytes_per_launch_full_workload: 1234\n")
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    assert bench.profiled_traffic("k.cu", "k.md") == 1234.0
    (csrc / "k.cu").write_text("// kernel v2\n")
    assert bench.profiled_traffic("k.cu", "k.md") is None
    assert bench.profiled_traffic("missing.cu", "k.md") is None


def test_resident_summary_gives_traffic_per_step_for_its_source():
    src = os.path.join(ROOT, "paper_1303_0107_gb300", "csrc", "resident.cu")
    summ = os.path.join(ROOT, "profiles", "resident_tree_2048x1024.md")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    t = bench.profiled_traffic("resident.cu", "resident_tree_2048x1024.md", "dram_bytes_per_step_full_workload")
    if os.path.exists(summ) and f"source_sha256_16: {h}" in open(summ).read():
        # the populations stay on chip: far below the 11.5 MB of algorithmic bytes per step
        assert t is not None and 0 <= t < 1e6
    else:
        assert t is None
