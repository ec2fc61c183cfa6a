"""CPU checks of the benchmark's DRAM-traffic figure (roofline.traffic): it
comes from a committed ncu capture and is reported only for the workload the
capture was taken on and only while the kernel sources are those captured."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _capture(root, digest, workload="c5"):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    d = {"kernels_sha256": digest,
         "kernels": {"k_cull_b": {"dram_bytes_read": 3.0e9, "dram_bytes_write": 1.0e9, "dram_bytes_per_launch": 4.0e9}}}
    json.dump(d, open(os.path.join(root, "profiles", f"traffic_{workload}.json"), "w"))


def test_traffic_reported_for_its_workload_and_sources(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _capture(str(tmp_path), bench.kernels_digest())
    assert bench.measured_traffic("k_cull_b", "c5") == 4.0e9
    assert bench.measured_traffic("k_cull_b", "c4") is None          # no capture of that workload
    assert bench.measured_traffic("k_cull_b", "c5_dmax50") is None   # nor of a range variant
    assert bench.measured_traffic("k_test", "c5") is None            # a kernel the capture does not cover


def test_traffic_null_once_the_kernels_change(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _capture(str(tmp_path), "0" * 64)
    assert bench.measured_traffic("k_cull_b", "c5") is None


def test_committed_capture_is_well_formed():
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic_c5.json")))
    assert len(d["kernels_sha256"]) == 64 and d["command"].startswith("ncu ")
    assert d["kernels"]
    for k, e in d["kernels"].items():
        assert e["dram_bytes_per_launch"] == e["dram_bytes_read"] + e["dram_bytes_write"] > 0


def test_digest_follows_code_not_comments(tmp_path):
    a = tmp_path / "k.cu"
    a.write_text("// kernel\n__global__ void k(float* x) { x[0] = 1.f; /* one */ }\n")
    d0 = bench.kernels_digest([str(a)])
    a.write_text("// the kernel, described differently\n__global__ void k(float* x) {\n  x[0] = 1.f;  // one\n}\n")
    assert bench.kernels_digest([str(a)]) == d0
    a.write_text("__global__ void k(float* x) { x[0] = 2.f; }\n")
    assert bench.kernels_digest([str(a)]) != d0
