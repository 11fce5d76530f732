"""Host logic of bench.py that feeds the JSON line's roofline: the DRAM traffic of the dominant stage is
read from the committed ncu summary only when that summary was captured from the current sources, and
then equals the sum of the stage's kernels in the table."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _table():
    rows = {}
    with open(bench.TRAFFIC_PROFILE) as f:
        for line in f:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if line.startswith("|") and cells[0].split(" ")[0].endswith("_kernel"):
                rows[cells[0].split(" ")[0]] = float(cells[3])
    return rows


def test_traffic_only_for_the_captured_sources(monkeypatch):
    with open(bench.TRAFFIC_PROFILE) as f:
        digest = next(line.split("`")[1] for line in f if line.startswith("Library source digest:"))
    table = _table()
    monkeypatch.setattr(bench, "library_digest", lambda: digest)
    for stage, kernels in bench.STAGE_KERNELS.items():
        got, note = bench.profiled_traffic(stage, "sparse512")
        assert got == pytest.approx(sum(table[k] for k in kernels) * 1e6), stage
        assert digest in note
    monkeypatch.setattr(bench, "library_digest", lambda: "0000000000000000")
    got, note = bench.profiled_traffic("rmsprop_step", "sparse512")
    assert got is None and "sources changed" in note
    assert bench.profiled_traffic("rmsprop_step", "sparse256")[0] is None

