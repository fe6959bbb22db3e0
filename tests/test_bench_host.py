"""Host-side pieces of bench.py that need no GPU: the algorithmic byte model
of the MIS-2 rounds and the rule that a DRAM-traffic record is used only
while the measured kernel's own sources are unchanged."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_round_byte_model_by_hand():
    # one round: W1 = 10 rows of D1 = 40 entries, W2 = 20 rows of D2 = 90
    # entries, n = 100, 4-byte rowptr
    n, s = 100, 4
    refresh = 8 * 10
    column = (8 + s) * 20 + 4 * 90 + 4 * min(n, 90 + 20)
    decide = (8 + s) * 10 + 4 * 40 + 4 * min(n, 40 + 10)
    compaction = 12 * (10 + 20)
    assert bench.mis2_bytes([[10, 20, 40, 90]], n, s) == refresh + column + decide + compaction
    # rounds add up; gathers are capped at one read of every vertex
    two = bench.mis2_bytes([[10, 20, 40, 90], [1000, 1000, 5000, 5000]], 500, 8)
    assert two == bench.mis2_bytes([[10, 20, 40, 90]], 500, 8) + bench.mis2_bytes([[1000, 1000, 5000, 5000]], 500, 8)
    assert bench.mis2_bytes(np.zeros((0, 4), dtype=np.int64), n, s) == 0


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    from paper_2204_02934_gb300 import _build

    files = ["device_loop.cu", "grid_sync.cuh", "internal.h", "mis_rows.cuh", "common.cuh", "mis2.h"]
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = prof / "k_test_traffic.txt"
    rec.write_text(f"kernel: k_test\nworkload_key: 27pt\ndram_bytes_per_launch: 1234\n"
                   f"source_files: {' '.join(files)}\nsource_digest: {_build.source_digest(files)}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_from_profile("k_test", "27pt") == 1234.0
    assert bench._traffic_from_profile("k_test", "rmat") is None  # taken on another workload
    rec.write_text(f"kernel: k_test\nworkload_key: 27pt\ndram_bytes_per_launch: 1234\n"
                   f"source_files: {' '.join(files)}\nsource_digest: 0000000000000000\n")
    assert bench._traffic_from_profile("k_test", "27pt") is None  # the kernel changed since the capture
    assert bench._traffic_from_profile("k_missing", "27pt") is None
