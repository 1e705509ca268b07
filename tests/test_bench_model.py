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
    """A capture's bytes scale by the launch's units while every listed
    source has the captured code digest; another graph, a changed source or
    a missing capture give None."""
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2512_11606_gb300", "csrc")
    digest = bench.code_digest(open(os.path.join(csrc, "ahpp_batch.cuh"), encoding="utf-8").read())
    rec = {"graph": "medium", "bytes_per_unit": 2.0, "l2_to_sm_bytes_per_unit": 3.0,
           "sources": {"ahpp_batch.cuh": digest}}
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"k_tiles": rec, "k_query1": dict(rec, bytes_per_unit=None)})
    assert bench.ncu_traffic("k_tiles", "medium", 10) == 20.0
    assert bench.ncu_traffic("k_tiles", "medium", 10, "l2_to_sm_bytes_per_unit") == 30.0
    assert bench.ncu_traffic("k_tiles", "tiny", 10) is None
    assert bench.ncu_traffic("k_query1", "medium", 10) is None
    bad = dict(rec, sources={"ahpp_batch.cuh": "0000000000000000"})
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"k_tiles": bad, "k_query1": bad})
    assert bench.ncu_traffic("k_tiles", "medium", 10) is None
    assert bench.ncu_traffic("k_tiles", "medium", 10, "l2_to_sm_bytes_per_unit") is None


class FakeServer:
    """Answers in submit order; records how many requests were outstanding
    at each submit."""

    def __init__(self):
        self.next, self.out, self.peak = 0, set(), 0
        self.args = {}

    def submit(self, q, eps, k):
        t = self.next
        self.next += 1
        self.out.add(t)
        self.peak = max(self.peak, len(self.out))
        self.args[t] = (q, eps, k)
        return t

    def wait(self, t, k):
        self.out.discard(t)
        q, eps, kk = self.args[t]
        assert kk == k

        class R:
            stats = {"served_ms": float(t), "rounds": q}
        return R


def test_closed_loop_keeps_the_backlog_and_order():
    srv = FakeServer()
    n, inflight = 100, 64
    qs = list(range(1000, 1000 + n))
    done_t, lat, rounds = bench.closed_loop(srv, qs, [1e-6] * n, [10 + i % 3 for i in range(n)], inflight)
    assert srv.peak == inflight and srv.next == n
    assert lat == [float(i) for i in range(n)] and rounds == qs
    assert all(b >= a for a, b in zip(done_t, done_t[1:]))
    s = bench.steady_state(done_t, lat, 40)
    assert s["window_queries"] == 20 and s["in_flight"] == 40
    assert bench.steady_state(done_t, lat, 48) is None


def test_steady_state_counts_whole_bursts():
    """Results of one server step arrive together: 32 every 5 ms is 6,400
    queries/s, whichever index the window would start and end at."""
    burst, period, n_bursts = 32, 5e-3, 40
    done_t = [b * period + j * 50e-6 for b in range(n_bursts) for j in range(burst)]
    lat = [1.0] * len(done_t)
    for inflight in (40, 47, 64, 70):
        s = bench.steady_state(done_t, lat, inflight)
        assert s["qps"] == pytest.approx(burst / period, rel=1e-9)
        assert s["window_queries"] % burst == 0
    # without the snapping, window edges inside bursts read off the rate
    lo, hi = 40, len(done_t) - 40
    assert abs((hi - lo) / (done_t[hi - 1] - done_t[lo - 1]) / (burst / period) - 1) > 0.005


def test_code_digest_ignores_comments_and_layout_only():
    src = 'int f(int x) {  // add one\n  /* body */ return x + 1;\n}\nconst char* s = "a // b";\n'
    same = 'int f(int x) { /* a different comment */\n\n    return x + 1; }\nconst char* s = "a // b"; // c\n'
    assert bench.code_digest(src) == bench.code_digest(same)
    assert bench.code_digest(src) != bench.code_digest(src.replace("x + 1", "x + 2"))
    assert bench.code_digest(src) != bench.code_digest(src.replace('"a // b"', '"a /* b"'))
    assert bench.code_digest("char c = '\\'';") != bench.code_digest("char c = '\\\\';")


def test_scaled_workloads_of_the_sweep():
    """The sweep's graphs: by nodes and edges (every size scaled, shapes kept)
    or by edges alone (same nodes, sparser), and the large recipe at F = 1."""
    from paper_2512_11606_gb300 import synth
    both = bench.graph_spec("large", 0.25)
    assert (both["n_u"], both["n_v"], both["n_e"], both["n_a"]) == (1_250_000, 1_250_000, 50_000_000, 12_500)
    edges = bench.graph_spec("large", 0.25, edges_only=True)
    assert (edges["n_u"], edges["n_v"], edges["n_e"], edges["n_a"]) == (5_000_000, 5_000_000, 50_000_000, 50_000)
    for spec in (both, edges):
        assert {k: spec[k] for k in ("m", "gamma_u", "gamma_v", "seed", "bf16")} == \
               {k: synth.LARGE[k] for k in ("m", "gamma_u", "gamma_v", "seed", "bf16")}
    assert bench.graph_spec("large") == synth.LARGE
