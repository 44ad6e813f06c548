"""The committed ncu summaries that bench.py reads its per-launch DRAM traffic
from: each names the figures the roofline line uses, and the reader returns
the traffic only while the summary's code hash matches the sources."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def fields(path):
    text = open(path).read()
    return dict(line.strip("- ").split(": ", 1) for line in text.splitlines()
                if line.startswith("- ") and ": " in line)


def test_each_summary_names_traffic_and_code_hash():
    for prec, path in bench.PROFILES.items():
        f = fields(path)
        assert int(f["traffic_bytes_per_launch"]) > 0, prec
        h = f["kernel_code_sha256_16"]
        assert len(h) == 16 and int(h, 16) >= 0, prec


def test_traffic_is_read_only_for_the_captured_code(monkeypatch):
    for prec, path in bench.PROFILES.items():
        f = fields(path)
        monkeypatch.setattr(bench, "kernel_fingerprint", lambda: f["kernel_code_sha256_16"])
        traffic, note = bench.profiled_traffic(prec)
        assert traffic == int(f["traffic_bytes_per_launch"]), note
        monkeypatch.setattr(bench, "kernel_fingerprint", lambda: "0" * 16)
        traffic, note = bench.profiled_traffic(prec)
        assert traffic is None and "changed" in note
