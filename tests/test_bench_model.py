"""The arithmetic behind bench.py's roofline fields, on CPU.

The byte model of a tile-round, the L2 row-access ceiling built from
measured rates, and the rule that drops the ncu traffic figure once the
kernel sources differ from the captured ones.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.argv = sys.argv[:1]
import bench  # noqa: E402

MEDIUM = dict(n_u=1_000_000, n_v=500_000, n_a=10_000, n_e=20_000_000, n_ea=20_000_000, batch_tile=32)


def test_round_bytes_medium_by_hand():
    nU, nV, nA, nE, nEA = 1_000_000, 500_000, 10_000, 20_000_000, 20_000_000
    graph = 16 * nE + 10 * nEA + 4 * (2 * (nU + 1) + nV + 1)           # three streamed directions
    state = 32 * 4 * (nU + nV + 2 * nA + nV + nA + 2 * nU + 4 * nU)   # per lane, per round
    assert bench.round_bytes(MEDIUM, 32) == graph + state
    assert 1.55e9 < bench.round_bytes(MEDIUM, 32) < 1.57e9
    # FP32 attribute weights add 2 bytes per U->A entry
    assert bench.round_bytes(MEDIUM, 32, bf16=False) - bench.round_bytes(MEDIUM, 32) == 2 * nEA


class FakeAhpp:
    """row_access_peak with fixed rates: gathers 80 G rows/s, reductions 50."""

    @staticmethod
    def row_access_peak(table_bytes, op, device):
        return 80e9 if op == "gather" else 50e9


def test_row_roofline_composes_the_measured_rates():
    tile_rounds, launch_s = 100, 0.15
    r = bench.row_roofline(FakeAhpp, MEDIUM, tile_rounds, launch_s, 0)
    t_min = 3 * 20e6 / 80e9 + 20e6 / 50e9          # 60 M gathers + 20 M reductions per tile-round
    assert r["frac"] == pytest.approx(tile_rounds * t_min / launch_s)
    assert r["rows_per_launch"] == tile_rounds * 80_000_000
    assert r["achieved"] == pytest.approx(r["rows_per_launch"] / launch_s)
    assert [p["table_bytes"] for p in r["parts"]] == [1_000_000 * 128, 500_000 * 128, 10_000 * 128,
                                                      10_000 * 128]


def test_ncu_traffic_applies_only_to_the_captured_sources(monkeypatch):
    assert bench.ncu_traffic("tiny", 10) is None
    good = dict(bench.NCU_TRAFFIC)
    bad = dict(good, sources=dict(good["sources"], **{"ahpp_batch.cu": "0000000000000000"}))
    monkeypatch.setattr(bench, "NCU_TRAFFIC", bad)
    assert bench.ncu_traffic("medium", 10) is None
    assert bench.ncu_traffic("medium", 10, "l2_to_sm_bytes_per_tile_round") is None
