"""Host-side pieces of bench.py that need no GPU: the DRAM traffic taken from
a committed ncu summary is used only while the kernel's sources are the ones
the counters were taken on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, sha, value):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / "s.md").write_text(f"Sources: a.cu with sha256 (of the two files concatenated) {sha}.\n"
                            f"traffic_bytes_per_launch: {value}\n")


def test_measured_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "a.cu"
    src.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.source_hash(["a.cu"])
    _summary(tmp_path, sha, 1234)
    assert bench.measured_traffic(["a.cu"], "s.md") == 1234
    src.write_text("__global__ void k() { }\n")           # the kernel changed since the capture
    assert bench.measured_traffic(["a.cu"], "s.md") is None
    assert bench.measured_traffic(["a.cu"], "missing.md") is None


def test_job_throughput_counts_every_rank():
    assert bench.job_throughput(1000, 4, 2.0) == 4 * 1000 / 2e-3
