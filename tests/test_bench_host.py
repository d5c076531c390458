"""Host logic of bench.py without a GPU: the roofline traffic guard (a DRAM figure from a committed
ncu summary is reported only while the kernel's sources still hash to the captured value) and the
algorithmic flop counts the roofline divides by."""
import hashlib
import json
import os

import bench


def _write_summary(path, sources, digest, traffic=12345):
    meta = {"kernel": "k", "traffic_bytes_per_launch": traffic, "sources": sources,
            "sources_sha256": digest}
    path.write_text("# summary\n\n<!-- traffic: " + json.dumps(meta) + " -->\n")


def test_traffic_guard_follows_the_source_hash(tmp_path, monkeypatch):
    pkg = os.path.join(bench.ROOT, "paper_1506_04448_gb300")
    sources = ["csrc/common.cuh", "csrc/fft.cuh"]
    digest = hashlib.sha256(b"".join(open(os.path.join(pkg, f), "rb").read() for f in sources)).hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    os.symlink(pkg, tmp_path / "paper_1506_04448_gb300")
    _write_summary(prof / "good.md", sources, digest)
    _write_summary(prof / "stale.md", sources, "0" * 64)
    assert bench.measured_traffic("good.md") == 12345
    assert bench.measured_traffic("stale.md") is None
    assert bench.measured_traffic("missing.md") is None


def test_algorithmic_flop_counts():
    # 5 b log2 b per length-b complex FFT; 4 per order-3 sketch-contraction, 2(p-1) for order p
    assert bench.fft_flops(14) == 5 * (1 << 14) * 14
    assert bench.contraction_flops(14) == 4 * 5 * (1 << 14) * 14
    assert bench.orderp_flops(12, 4) == 6 * 5 * (1 << 12) * 12
