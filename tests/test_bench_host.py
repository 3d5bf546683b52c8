"""Host-side logic of bench.py that decides what the JSON line reports: the
recorded DRAM traffic is used only while the kernel's code is unchanged."""
import json

import pytest

import bench


def test_source_hash_ignores_comments_and_layout(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2006_09299_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (csrc / "k.cu").write_text("int f(int a) {\n    return a + 1;   // one more\n}\n")
    h0 = bench.kernel_source_hash("k.cu")
    (csrc / "k.cu").write_text("/* block\n comment */ int f(int a) { return a + 1; }  // changed comment\n\n")
    assert bench.kernel_source_hash("k.cu") == h0
    (csrc / "k.cu").write_text("int f(int a) {\n    return a + 2;\n}\n")
    assert bench.kernel_source_hash("k.cu") != h0


def test_recorded_traffic_scales_and_goes_stale(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2006_09299_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (csrc / "k.cu").write_text("int f(int a) { return a; }\n")
    rec = {"k.cu": {"file": "k.cu", "source_sha256_16": bench.kernel_source_hash("k.cu"),
                    "dram_bytes_per_pixel": {"sweep4096": 9.5}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("k.cu", "sweep4096", 1000) == pytest.approx(9500.0)
    assert bench.recorded_traffic("k.cu", "rings8192", 1000) is None      # not captured there
    (csrc / "k.cu").write_text("int f(int a) { return -a; }\n")
    assert bench.recorded_traffic("k.cu", "sweep4096", 1000) is None      # code changed since



def test_source_hash_follows_local_headers(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2006_09299_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (csrc / "dev.cuh").write_text("inline int g(int a) { return a; }\n")
    (csrc / "k.cu").write_text('#include "dev.cuh"\n#include <cstdint>\nint f(int a) { return g(a); }\n')
    h0 = bench.kernel_source_hash("k.cu")
    (csrc / "dev.cuh").write_text("inline int g(int a) { return a; }   // comment only\n")
    assert bench.kernel_source_hash("k.cu") == h0
    (csrc / "dev.cuh").write_text("inline int g(int a) { return a + 1; }\n")
    assert bench.kernel_source_hash("k.cu") != h0          # a header edit makes the record stale


def test_full_output_roofline_counts_labels_and_node_records():
    """9 B/px for the path (8 B/px for the writer) plus 60 B per node."""
    r = bench.full_output_roofline(px=1000, nodes=10, path_ms=1e-3, write_ms=2e-3, peak=100.0, peak_kind="measured")
    assert r["bytes_per_node"] == 60 and r["nodes"] == 10
    assert r["path"]["algorithmic_bytes"] == 9 * 1000 + 60 * 10
    assert r["k_write"]["algorithmic_bytes"] == 8 * 1000 + 60 * 10
    # bytes / (ms * 1e-3) / 1e9 GB/s
    assert r["path"]["achieved"] == pytest.approx(9600 / 1e-6 / 1e9, rel=1e-3)
    assert r["k_write"]["frac"] == pytest.approx(8600 / 2e-6 / 1e9 / 100.0, rel=1e-3)
    assert "k_write" not in bench.full_output_roofline(1000, 10, 1e-3, None, 100.0, "measured")
