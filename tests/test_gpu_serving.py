"""Serving loop (continuous batching) through the C ABI.

Requests of different eps and k arrive while others are on the device; they
are admitted into free slots of tiles already in flight.  Every sampled
result must equal the same query alone (its dense vector, element by element
within 1e-6) and the FP64 oracle push (within 1e-6), with top-k overlap
>= 0.99 under the 2 eps tie rule; requests with k = |U| return the whole
vector, which is compared element by element over all of U.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2512_11606_gb300 import synth
from parity_util import check_dense, check_topk

pytestmark = pytest.mark.gpu
ALPHA, BETA = 0.15, 0.35
TOL = 1e-6


@pytest.fixture(scope="module")
def ahpp():
    from paper_2512_11606_gb300 import build
    build.build()
    from paper_2512_11606_gb300 import ahpp as mod
    return mod


@pytest.fixture(scope="module")
def tiny(ahpp):
    g = synth.make_graph(**synth.TINY)
    og = oracle.OracleGraph.from_arrays(g)
    lam, _ = og.lambda_estimate(ALPHA, BETA)
    G = ahpp.Graph.from_arrays(g, lam=lam, attr_bf16=0)
    yield dict(g=g, og=og, lam=lam, G=G)
    G.close()


def check_same(G, res, q, eps, k):
    """A served result against the same query alone (the plain path's dense
    reserve vector): every returned score within 1e-6, a valid top-k."""
    alone, st, rc = G.query_dense(int(q), float(eps))
    assert rc == 0
    check_topk(res.nodes, res.scores, alone, k, float(eps))
    assert res.stats["rounds"] == st["rounds"]
    return alone


def as_dense(res, n_u):
    """The whole vector of a result with k = |U| (every node, once)."""
    out = np.full(n_u, np.nan)
    out[res.nodes] = res.scores
    assert not np.isnan(out).any()
    return out


def test_served_results_equal_alone_in_a_mix(ahpp, tiny):
    G, og, lam = tiny["G"], tiny["og"], tiny["lam"]
    rng = np.random.default_rng(3)
    n = 90
    qs = synth.draw_queries(tiny["g"].n_u, n, seed=31)
    eps = np.exp(rng.uniform(np.log(1e-7), np.log(1e-4), n))
    ks = rng.choice([10, 100, 1000], n)         # the serving workload's k mix
    n_u = tiny["g"].n_u
    ks[[1, 41, 77]] = n_u                       # whole vectors, compared over all of U
    srv = ahpp.Server(G, max_slots=64, rounds_per_step=2)
    try:
        # first wave, then more requests while the first ones are in flight
        tickets = [srv.submit(int(qs[i]), float(eps[i]), int(ks[i])) for i in range(40)]
        first = srv.wait(tickets[0], int(ks[0]))
        assert first is not None
        tickets += [srv.submit(int(qs[i]), float(eps[i]), int(ks[i])) for i in range(40, n)]
        info = srv.info()
        assert info["submitted"] == n and info["slots"] == 64
        results = [first] + [srv.wait(t, int(k)) for t, k in zip(tickets[1:], ks[1:])]
        info = srv.info()
        assert info["completed"] == n and info["in_flight"] == 0 and info["queued"] == 0
        assert info["steps"] >= 2
    finally:
        srv.stop()
    for i in [0, 1, 39, 40, 41, 77, 89]:
        r = results[i]
        assert r.rc == 0 and r.stats["status"] == 0
        alone = check_same(G, r, qs[i], eps[i], int(ks[i]))
        ref = og.push("asrp", ALPHA, BETA, int(qs[i]), float(eps[i]), lam=lam)
        check_topk(r.nodes, r.scores, ref.pi, int(ks[i]), float(eps[i]))
        assert abs(r.stats["rounds"] - ref.stats["rounds"]) <= 1
        if ks[i] == n_u:
            full = as_dense(r, n_u)
            check_dense(full, alone)
            check_dense(full, ref.pi)


def test_admission_while_in_flight(ahpp, tiny):
    """Slots free up and are refilled while other slots of the same tile run."""
    G = tiny["G"]
    srv = ahpp.Server(G, max_slots=32, rounds_per_step=1)
    try:
        qs = synth.draw_queries(tiny["g"].n_u, 64, seed=41)
        # loose eps finish in a few rounds, tight ones take many: the loose
        # ones' slots are reused while the tight ones are still running
        eps = [1e-3 if i % 2 else 1e-8 for i in range(64)]
        t = [srv.submit(int(q), e, 5) for q, e in zip(qs, eps)]
        seen_mix = False
        for _ in range(2000):
            info = srv.info()
            if info["completed"] > 0 and info["in_flight"] > 0 and info["completed"] + info["in_flight"] > 32:
                seen_mix = True
                break
            time.sleep(0.001)
        res = [srv.wait(x, 5) for x in t]
        assert all(r is not None and r.rc == 0 for r in res)
        assert seen_mix
    finally:
        srv.stop()


def test_queue_full_and_bad_requests(ahpp, tiny):
    G = tiny["G"]
    srv = ahpp.Server(G, max_slots=32, queue_capacity=2, rounds_per_step=8)
    try:
        got, busy = [], 0
        for q in synth.draw_queries(tiny["g"].n_u, 200, seed=51):
            t = srv.try_submit(int(q), 1e-8, 10)
            if t is None:
                busy += 1
            else:
                got.append(t)
        assert busy > 0 and srv.info()["rejected"] == busy
        with pytest.raises(ahpp.AhppError) as e:
            srv.submit(tiny["g"].n_u, 1e-6, 10)
        assert e.value.code == ahpp.AHPP_EINVAL
        with pytest.raises(ahpp.AhppError):
            srv.submit(0, -1.0, 10)
        for t in got:
            assert srv.wait(t, 10).rc == 0
        with pytest.raises(ahpp.AhppError) as e:
            srv.wait(got[0], 10)          # delivered once
        assert e.value.code == ahpp.AHPP_EINVAL
    finally:
        srv.stop()


def test_hbm_budget_limits_slots(ahpp, tiny):
    g = tiny["g"]
    G = ahpp.Graph.from_arrays(g, lam=tiny["lam"], attr_bf16=0)
    info = G.info
    G.close()
    used = info["graph_bytes"] + info["query_state_bytes"]
    per_tile_lower = g.n_u * 32 * 12            # residues, reserves, compensation of one tile
    room = 12_000_000
    G = ahpp.Graph.from_arrays(g, lam=tiny["lam"], attr_bf16=0, hbm_budget_bytes=used + room)
    try:
        srv = ahpp.Server(G)
        slots = srv.info()["slots"]
        srv.stop()
        assert 32 <= slots and (slots // 32) * per_tile_lower <= room
    finally:
        G.close()
    G = ahpp.Graph.from_arrays(g, lam=tiny["lam"], attr_bf16=0, hbm_budget_bytes=used + 100_000)
    try:
        with pytest.raises(ahpp.AhppError) as e:
            ahpp.Server(G)
        assert e.value.code == ahpp.AHPP_ENOMEM
    finally:
        G.close()


def test_served_latency_is_reported(ahpp, tiny):
    srv = ahpp.Server(tiny["G"], max_slots=32)
    try:
        t = srv.submit(5, 1e-6, 10)
        r = srv.wait(t, 10)
        assert r.stats["served_ms"] > 0
    finally:
        srv.stop()


def test_served_app_equals_alone_and_oracle(ahpp, tiny):
    """Serving with APP (Algorithm 3): per-request eps, each served result is
    the query alone and the oracle's APP push."""
    g, og = tiny["g"], tiny["og"]
    G = ahpp.Graph.from_arrays(g, algo=ahpp.AHPP_APP, attr_bf16=0)
    try:
        qs = synth.draw_queries(g.n_u, 40, seed=81)
        eps = [1e-6 if i % 2 else 1e-4 for i in range(40)]
        srv = ahpp.Server(G, max_slots=32, rounds_per_step=3)
        try:
            t = [srv.submit(int(q), e, 50) for q, e in zip(qs, eps)]
            res = [srv.wait(x, 50) for x in t]
        finally:
            srv.stop()
        for i in [0, 1, 31, 32, 39]:
            r = res[i]
            assert r.rc == 0 and r.stats["status"] == 0
            check_same(G, r, qs[i], eps[i], 50)
            ref = og.push("app", ALPHA, BETA, int(qs[i]), eps[i])
            check_topk(r.nodes, r.scores, ref.pi, 50, eps[i])
    finally:
        G.close()


def test_light_load_uses_the_single_query_path(ahpp, tiny):
    """With nothing running and a short queue the server answers on the
    single-query path (the plain query's kernel, equal up to the order of its
    FP32 atomic sums).  With the single path disabled the same request goes
    through a tile and matches within the tolerance."""
    G = tiny["G"]
    q, eps, k = 17, 1e-6, 20
    alone = G.query(q, eps, k)
    srv = ahpp.Server(G, max_slots=32)
    try:
        r = srv.wait(srv.submit(q, eps, k), k)
    finally:
        srv.stop()
    check_same(G, r, q, eps, k)
    assert r.stats["served_ms"] > 0
    assert r.stats["dense_rounds"] == alone.stats["dense_rounds"]   # the plain path's push/pull split
    srv = ahpp.Server(G, max_slots=32, single_max=-1)
    try:
        r2 = srv.wait(srv.submit(q, eps, k), k)
    finally:
        srv.stop()
    check_same(G, r2, q, eps, k)


def test_cancel_queued_and_in_flight(ahpp, tiny):
    """A cancelled queued request and a cancelled request on the device both
    end with AHPP_ECANCELED (or their result if they finished first); the
    other requests are unaffected and equal the query alone."""
    G = tiny["G"]
    srv = ahpp.Server(G, max_slots=32, rounds_per_step=1, single_max=-1)
    try:
        qs = synth.draw_queries(tiny["g"].n_u, 80, seed=91)
        t = [srv.submit(int(q), 1e-8, 10) for q in qs]     # 32 on the device, 48 queued
        assert srv.cancel(t[70]) == 0                        # still queued
        for _ in range(2000):                                # wait until the first slots run
            if srv.info()["in_flight"] > 0:
                break
            time.sleep(0.001)
        assert srv.cancel(t[3]) == 0                         # on the device (or already done)
        res = {i: srv.wait(t[i], 10) for i in range(80)}
        assert res[70].rc == ahpp.AHPP_ECANCELED and res[70].nodes.shape[0] == 0
        assert res[3].rc in (ahpp.AHPP_ECANCELED, 0)
        with pytest.raises(ahpp.AhppError):
            srv.cancel(t[5])                                 # delivered already
        info = srv.info()
        assert info["in_flight"] == 0 and info["queued"] == 0
    finally:
        srv.stop()
    for i in (0, 4, 40, 79):
        assert res[i].rc == 0
        check_same(G, res[i], qs[i], 1e-8, 10)
