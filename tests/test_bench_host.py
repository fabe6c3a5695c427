"""Host-side logic of bench.py that needs no GPU: the smaller case of a workload (--objects) keeps the first objects
of the full one, the reported loss-curve steps, and the source hash that ties committed DRAM figures to the kernel
code (comment edits keep it, code edits change it)."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def bench(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    import bench as b
    yield b
    b.WORKLOAD_KEY, b.WORKLOAD = "multi8", b.WORKLOADS["multi8"]


def test_objects_override_keeps_the_first_objects(bench):
    full = bench.WORKLOADS["uneven32"]
    small = dict(full, objects=8)
    assert bench.workload_rays(small) == bench.workload_rays(full)[:8]
    bench.WORKLOAD_KEY, bench.WORKLOAD = "uneven32", small
    assert bench.workload_id() == "uneven32:objects=8"
    bench.WORKLOAD = full
    assert bench.workload_id() == "uneven32"


def test_curve_steps(bench):
    steps = bench.curve_steps(200)
    assert steps[0] == 0 and steps[-1] == 199 and len(steps) == 11 and steps == sorted(set(steps))
    assert bench.curve_steps(5) == [0, 1, 2, 3, 4]


def test_kernel_source_hash_ignores_comments(bench, tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_2304_05735_gb300", "csrc")
    dst = tmp_path / "paper_2304_05735_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash("mixed")
    f = dst / bench.KERNEL_SOURCES["mixed"][0]
    text = f.read_text()
    f.write_text("// a comment line\n" + text.replace("\n", "  // trailing comment\n", 1) + "\n\n")
    assert bench.kernel_source_hash("mixed") == h0
    f.write_text(text + "\nstatic const int kProbe = 1;\n")
    assert bench.kernel_source_hash("mixed") != h0


def test_profiled_traffic_needs_matching_source_and_workload(bench, tmp_path, monkeypatch):
    import json

    (tmp_path / "profiles").mkdir()
    shutil.copytree(os.path.join(ROOT, "paper_2304_05735_gb300", "csrc"),
                    tmp_path / "paper_2304_05735_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("mixed")
    entry = {"source_hash": h, "bytes_per_launch_full_workload": 1234}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps({"k_tile_tc|mixed|multi8": entry}))
    bench.WORKLOAD_KEY, bench.WORKLOAD = "multi8", bench.WORKLOADS["multi8"]
    assert bench.profiled_traffic("k_tile_tc", "mixed") == 1234
    bench.WORKLOAD_KEY, bench.WORKLOAD = "uneven32", bench.WORKLOADS["uneven32"]
    assert bench.profiled_traffic("k_tile_tc", "mixed") is None
    entry["source_hash"] = "0" * 16
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps({"k_tile_tc|mixed|multi8": entry}))
    bench.WORKLOAD_KEY, bench.WORKLOAD = "multi8", bench.WORKLOADS["multi8"]
    assert bench.profiled_traffic("k_tile_tc", "mixed") is None
