"""Host logic of bench.py that needs no GPU: the DRAM-traffic key of the
roofline (read from profiles/leaf_traffic.json; reported only for the
configuration it was measured on and only while the leaf sources are the ones
it was measured on), and the command line."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_key_matches_committed_sources():
    t = bench.leaf_traffic(1, 8192, 8192, 1, 6)
    if t is None:  # the bench then reports no traffic; the summary needs a new capture
        pytest.skip("leaf DRAM summary was measured on other sources")
    assert isinstance(t, int) and t > 2_000_000_000  # at least the algorithmic 2.3 GB


@pytest.mark.parametrize("cfg", [(2, 8192, 8192, 1, 3), (1, 4096, 4096, 1, 6), (1, 8192, 8192, 2, 6),
                                 (1, 8192, 8192, 1, 5)])
def test_traffic_only_for_the_measured_configuration(cfg):
    assert bench.leaf_traffic(*cfg) is None


def test_traffic_file_names_its_profile_summaries():
    import json
    with open(os.path.join(ROOT, "profiles", "leaf_traffic.json")) as f:
        caps = json.load(f)["captures"]
    for c in caps:
        assert os.path.exists(os.path.join(ROOT, "profiles", c["summary"]))


def test_traffic_dropped_when_a_leaf_source_changes(tmp_path, monkeypatch):
    """A copy of the tree whose leaf kernel differs by one byte reports no
    traffic: the summary was measured on other sources."""
    root = tmp_path / "tree"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "profiles", "leaf_traffic.json"), root / "profiles")
    src = root / "paper_2110_13042_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in ("leaf_tc.cu", "ptx.cuh", "plan.cpp"):
        shutil.copy(os.path.join(ROOT, "paper_2110_13042_gb300", "csrc", name), src / name)
    expected = bench.leaf_traffic(1, 8192, 8192, 1, 6)
    if expected is None:
        pytest.skip("leaf DRAM summary was measured on other sources")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.leaf_traffic(1, 8192, 8192, 1, 6) == expected  # same sources: same key
    with open(src / "leaf_tc.cu", "a") as f:
        f.write("\n")
    assert bench.leaf_traffic(1, 8192, 8192, 1, 6) is None


def test_command_line_modes():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True,
                         text=True, check=True).stdout
    for flag in ("--gpus", "--steps", "--warmup", "--impl", "--mode", "--batched-only", "--no-extras"):
        assert flag in out
    for mode in ("f64_emu", "f64", "f32", "f32_bf16", "f32_fp8"):
        assert mode in out
