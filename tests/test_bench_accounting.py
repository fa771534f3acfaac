"""The benchmark's accounting (CPU only): algorithmic bytes and flops per
site as the design notes derive them, the workload description both arms
print, and the traffic figure withheld once the kernel sources change."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import bench  # noqa: E402


def test_algorithmic_bytes_and_flops():
    # per output site and hop: input spinor + output spinor + 8 links
    assert bench.hop_bytes("f64", 18) == (24 + 24 + 8 * 18) * 8 == 1536
    assert bench.hop_bytes("f64", 12) == 1152
    assert bench.hop_bytes("f32", 12) == 576
    assert bench.hop_bytes("f16", 12) == 288 + 8           # the two per-site norms
    # Q_tm per even site: two hops + the re-read of psi_e in the second launch
    assert bench.algo_bytes("f64", 18)["qtm"] == 2 * 1536 + 192 == 3264
    assert bench.HOP_FLOPS == 1320
    assert bench.QTM_FLOPS == 2 * 1320 + 72 + 96 == 2808


def test_workload_config_names_the_workload():
    c = bench.workload_config((32, 32, 32, 64), "f64", 18, 1)
    assert c["lattice"] == [32, 32, 32, 64] and c["even_sites"] == 1048576
    assert c["bytes_per_step"] == 1048576 * 3264
    assert c["flops_per_step"] == 1048576 * 2808
    assert "32x32x32x64" in c["workload"] and "replicas" in c["parallelism"]


def test_traffic_only_for_the_captured_sources(monkeypatch):
    vh = 1048576
    if bench.kernel_source_hash() == bench.TRAFFIC["src"]:
        t = bench.traffic_per_launch("f64", 18, vh)
        # DRAM bytes of launch B: at least the compulsory read, not wildly above it
        assert bench.algo_bytes("f64", 18)["kernel_b"] * vh * 0.9 < t < 1.2 * 1800 * vh
    monkeypatch.setitem(bench.TRAFFIC, "src", "not-these-sources")
    assert bench.traffic_per_launch("f64", 18, vh) is None
    assert bench.traffic_per_launch("f64", 12, vh) is None
