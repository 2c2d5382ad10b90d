"""Host-side helpers of bench.py (no GPU): the committed ncu traffic summary is self-consistent
and is used only while the step kernels' sources match the hash it was taken on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def read_summary():
    d = {}
    with open(os.path.join(ROOT, "profiles", "k_step_f32_traffic.txt")) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                d[k.strip()] = v.strip()
    return d


def test_traffic_summary_is_consistent():
    d = read_summary()
    per_node = float(d["dram_bytes_per_launch"]) / int(d["pure_tile_nodes"])
    assert abs(per_node - float(d["dram_bytes_per_pure_node"])) < 1e-3
    # the capture moved the algorithmic bytes of the FP32 pure tiles to within 1 %
    assert abs(per_node / int(d["algorithmic_bytes_per_pure_node"]) - 1.0) < 0.01
    assert len(d["source_sha256_16"]) == 16


def test_traffic_is_reported_only_for_the_hashed_sources(monkeypatch):
    d = read_summary()
    nodes = 7165952
    expected = float(d["dram_bytes_per_pure_node"]) * nodes
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: d["source_sha256_16"])
    assert bench.profiled_traffic(nodes) == expected
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic(nodes) is None
