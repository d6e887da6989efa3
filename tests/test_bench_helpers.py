"""Host-side helpers of bench.py (no GPU): the workload's name, the lookup of
the committed DRAM-traffic figure by kernel source hash and workload, and the
serving ratio reported at the top level."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workload_named_by_the_scale_it_ran_at():
    assert bench.workload_label(bench.parse_args([])) == "rmat22"
    assert bench.workload_label(bench.parse_args(["--rmat-scale", "21"])) == "rmat21"
    assert bench.workload_label(bench.parse_args(["--workload", "road1m"])) == "road1m"


def test_traffic_reported_only_for_its_kernel_and_workload(tmp_path):
    good = bench.profiled_traffic("rmat22")
    assert good is not None and good > 0          # the committed summary matches the sources
    assert bench.profiled_traffic("rmat21") is None
    stale = tmp_path / "t.txt"
    stale.write_text("workload=rmat22\nkernel_source_hash=0000000000000000\n"
                     "dram_bytes_per_launch=5\n")
    assert bench.profiled_traffic("rmat22", str(stale)) is None
    fresh = tmp_path / "f.txt"
    fresh.write_text(f"workload=rmat22\nkernel_source_hash={bench.kernel_source_hash()}\n"
                     "dram_bytes_per_launch=5\n")
    assert bench.profiled_traffic("rmat22", str(fresh)) == 5.0


def test_kernel_source_hash_ignores_comments(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2608_21826_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text("int x; // one\n/* two */ int y;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_source_hash(("a.cu",))
    (csrc / "a.cu").write_text("int x; // changed comment\n/* other */ int y;\n")
    assert bench.kernel_source_hash(("a.cu",)) == h1
    (csrc / "a.cu").write_text("int x; int z;\n")
    assert bench.kernel_source_hash(("a.cu",)) != h1


def test_serve_min_ratio_over_half_load_and_above():
    rates = [{"fraction_of_batched_saturation": f, "served_qps": s, "plain_qps": 1.0}
             for f, s in ((0.25, 1.5), (0.5, 2.7), (0.75, 2.9), (1.1, 2.8))]
    assert bench._serve_min_ratio({"rates": rates}) == 2.7
    assert bench._serve_min_ratio(None) is None
