"""Host logic of bench.py that needs no GPU: the units a kernel's DRAM traffic scales with, and
the profile tables of DRAM bytes and warp instructions per unit (read only while the kernel's
sources are unchanged)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

FRAME = {"n_in_frustum": 1000, "n_mlp_queries": 900, "n_survivors": 600, "n_pairs": 5000, "sort_passes": 6}


def test_kernel_units():
    assert bench.kernel_units("k_mlp_tc", FRAME) == 900
    assert bench.kernel_units("k_blend<16>", FRAME) == 5000
    assert bench.kernel_units("k_project", FRAME) == 600
    # four 8-bit passes over the survivors' depth keys (32-bit), the rest over the pairs' tile keys
    # (16-bit up to 65536 tiles, else 32-bit in the same kernels as the depth passes)
    assert bench.kernel_units("k_rs_scatter<u32>", FRAME) == 4 * 600
    assert bench.kernel_units("k_rs_scatter<u16>", FRAME) == 2 * 5000
    assert bench.kernel_units("k_rs_hist<u16>", FRAME) == 2 * 5000
    assert bench.kernel_units("k_rs_scatter<u32>", FRAME, tile16=False) == 4 * 600 + 2 * 5000
    assert bench.kernel_units("k_frustum", FRAME) is None


def test_traffic_table_scaling_and_staleness(tmp_path, monkeypatch):
    h = bench.sources_hash("k_mlp_tc")
    table = tmp_path / "t.txt"
    table.write_text("| kernel | unit | bytes | hash |\n|---|---|---:|---|\n"
                     f"| `k_mlp_tc` | query | 24.5 | `{h}` |\n"
                     "| `k_project` | survivor | 300.0 | `0000000000000000` |\n")
    monkeypatch.setattr(bench, "TRAFFIC_TABLE", str(table))
    # bytes per unit x units of the frames / launches
    assert bench.dram_traffic_per_launch("k_mlp_tc", [FRAME, FRAME], 2) == pytest.approx(24.5 * 900)
    # a recorded hash that no longer matches the sources: null
    assert bench.dram_traffic_per_launch("k_project", [FRAME], 1) is None
    # no row, no sources list: null
    assert bench.dram_traffic_per_launch("k_blend<16>", [FRAME], 1) is None
    assert bench.dram_traffic_per_launch("k_frustum", [FRAME], 1) is None



def test_issue_table_is_read_only_while_sources_match(tmp_path, monkeypatch):
    h = bench.sources_hash("k_blend<16>")
    table = tmp_path / "i.txt"
    table.write_text("| kernel | unit | warp instructions per unit | hash |\n|---|---|---:|---|\n"
                     f"| `k_blend<16>` | evaluation | 1.085 | `{h}` |\n"
                     "| `k_project` | survivor | 40.0 | `0000000000000000` |\n")
    monkeypatch.setattr(bench, "ISSUE_TABLE", str(table))
    assert bench.issue_per_unit("k_blend<16>") == pytest.approx(1.085)
    assert bench.issue_per_unit("k_project") is None     # stale hash
    assert bench.issue_per_unit("k_mlp_tc") is None      # no row
    assert bench.issue_per_unit("k_frustum") is None     # no sources list
