"""Parity at the full workload sizes, in the launch configuration bench.py times.

Medium (|U|=1M, |V|=500k, |E|=20M, |A|=10k x 20, bf16 attribute weights):
one query is compared element by element with the FP64 oracle push (the
oracle takes about half a minute), and the same query inside a 64-query
batched launch (two tiles, bench's kernel and grid) is compared with both.
Every query of the batch is checked for properties that hold at any size.

Large (|U|=|V|=5M, |E|=200M, |A|=50k x 30, 256-query batch, top-1,000):
too big for the oracle's exact push in a test, so it is checked through
properties that hold at any size: mass conservation, nonnegativity, the
batched result equal to the result alone, and top-k consistent with the
reserves; Theorem 2 against the GPU's Algorithm 1; and serving with the
serving workload's request mix.  Generating that graph takes minutes on the
host, so the test runs only with AHPP_LARGE=1.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2512_11606_gb300 import synth

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
def medium(ahpp):
    g = synth.make_graph(**synth.MEDIUM_BF16)
    og = oracle.OracleGraph.from_arrays(g)
    lam, _ = og.lambda_estimate(ALPHA, BETA)
    G = ahpp.Graph.from_arrays(g, lam=lam)
    yield dict(g=g, og=og, lam=lam, G=G)
    G.close()


def test_medium_lambda_on_gpu_matches_oracle(ahpp, medium):
    G2 = ahpp.Graph.from_arrays(medium["g"])
    lam_gpu = G2.lam
    G2.close()
    assert lam_gpu >= medium["lam"] * (1 - 1e-6)
    assert abs(lam_gpu - medium["lam"]) / medium["lam"] <= 2e-4


def test_medium_single_and_batched_vs_oracle(medium):
    G, og, lam, g = medium["G"], medium["og"], medium["lam"], medium["g"]
    q1024 = [int(x) for x in synth.draw_queries(g.n_u, 1024)]
    qs = q1024[:64]
    q = qs[0]
    eps = 1e-6
    ref = og.push("asrp", ALPHA, BETA, q, eps, lam=lam)
    alone, st, rc = G.query_dense(q, eps)
    assert rc == 0
    assert np.abs(alone.astype(np.float64) - ref.pi).max() <= TOL
    assert abs(st["rounds"] - ref.stats["rounds"]) <= 1
    dense, stats, rc = G.query_batch_dense(qs, eps)
    assert rc == 0
    assert np.abs(dense[0].astype(np.float64) - ref.pi).max() <= TOL
    assert np.abs(dense[0] - alone).max() <= TOL
    for i in range(len(qs)):
        s = stats[i]
        assert s["status"] == 0 and s["mass_err"] < 1e-5
        assert dense[i].min() >= 0.0 and dense[i][qs[i]] >= ALPHA - TOL
        assert s["max_resid"] <= s["eps_f"] * (1 + 1e-6)
        assert s["eps_f"] <= eps / lam * (1 + 1e-6)

    # the eps guarantee of Theorem 2 against the GPU's Algorithm 1 at T = 250
    # ((1 - alpha)^250 < 1e-17): 0 <= pi - pi_hat <= eps, up to FP32 rounding
    for i in (0, 63):
        pi_T, _, rc = G.power_iteration(qs[i], 250)
        assert rc == 0
        d = pi_T.astype(np.float64) - dense[i].astype(np.float64)
        assert d.min() >= -5e-7 and d.max() <= eps + 5e-7
        if i == 0:
            assert np.abs(pi_T.astype(np.float64) - ref.pi).max() <= eps + TOL

    # the launch bench.py times: 1,024 queries, top-100 each
    k = 100
    res = G.query_batch(q1024, eps, k)
    assert all(r.rc == 0 and r.stats["status"] == 0 for r in res)
    top = res[0]
    assert top.nodes.shape[0] == k
    assert np.all(np.diff(top.scores) <= 0)
    assert np.abs(top.scores.astype(np.float64) - ref.pi[top.nodes]).max() <= TOL
    kth = np.sort(ref.pi)[-k]
    assert ref.pi[top.nodes].min() >= kth - 2 * TOL      # a valid top-k of the oracle's scores
    for i in range(1, 64):
        r = res[i]
        assert np.abs(r.scores - dense[i][r.nodes]).max() <= TOL
        kth_i = np.sort(dense[i])[-k]
        assert dense[i][r.nodes].min() >= kth_i - 2 * TOL


@pytest.mark.parametrize("eps", [1e-5, 1e-7])
def test_medium_single_query_other_eps(medium, eps):
    """The single-query workload's other error thresholds: every score within
    1e-6 of the oracle push, top-100 overlap with the oracle >= 0.99."""
    G, og, lam, g = medium["G"], medium["og"], medium["lam"], medium["g"]
    q = int(synth.draw_queries(g.n_u, 2, seed=7)[1])
    ref = og.push("asrp", ALPHA, BETA, q, eps, lam=lam)
    pi, st, rc = G.query_dense(q, eps)
    assert rc == 0 and st["status"] == 0
    assert np.abs(pi.astype(np.float64) - ref.pi).max() <= max(TOL, eps)
    assert abs(st["rounds"] - ref.stats["rounds"]) <= 1
    top = G.query(q, eps, 100)
    order = np.lexsort((np.arange(g.n_u), -ref.pi))
    kth = ref.pi[order[99]]
    ok = set(np.nonzero(ref.pi >= kth - 2 * max(eps, TOL))[0].tolist())
    assert len(set(top.nodes.tolist()) & ok) / 100 >= 0.99


def test_medium_served_mix_equals_alone(ahpp, medium):
    """Continuous batching at full size with the serving workload's request
    mix (eps log-uniform in [1e-7, 1e-4], k in {10, 100, 1000}): requests
    admitted while others run give the same result as the query alone, and
    one of them is checked against the oracle."""
    G, og, lam, g = medium["G"], medium["og"], medium["lam"], medium["g"]
    rng = np.random.default_rng(17)
    n = 48
    qs = synth.draw_queries(g.n_u, n, seed=61)
    eps = np.exp(rng.uniform(np.log(1e-7), np.log(1e-4), n))
    ks = rng.choice([10, 100, 1000], n)
    srv = ahpp.Server(G, max_slots=32, rounds_per_step=8)
    try:
        tickets = [srv.submit(int(qs[i]), float(eps[i]), int(ks[i])) for i in range(24)]
        first = srv.wait(tickets[0], int(ks[0]))
        tickets += [srv.submit(int(qs[i]), float(eps[i]), int(ks[i])) for i in range(24, n)]
        results = [first] + [srv.wait(t, int(k)) for t, k in zip(tickets[1:], ks[1:])]
        info = srv.info()
        assert info["completed"] == n and info["steps"] > 1
    finally:
        srv.stop()
    for i in [0, 5, 23, 24, 30, 47]:
        r = results[i]
        assert r.rc == 0 and r.stats["status"] == 0 and r.stats["mass_err"] < 1e-5
        alone = G.query(int(qs[i]), float(eps[i]), int(ks[i]))
        assert r.stats["rounds"] == alone.stats["rounds"]
        common = len(set(r.nodes.tolist()) & set(alone.nodes.tolist())) / int(ks[i])
        assert common >= 0.98
        a = dict(zip(alone.nodes.tolist(), alone.scores.tolist()))
        assert all(abs(sc - a[v]) <= TOL for v, sc in zip(r.nodes.tolist(), r.scores.tolist()) if v in a)
    i = int(np.argmin(eps[:24]))                  # the tightest eps of the first wave
    ref = og.push("asrp", ALPHA, BETA, int(qs[i]), float(eps[i]), lam=lam)
    r = results[i]
    assert np.abs(r.scores.astype(np.float64) - ref.pi[r.nodes]).max() <= TOL


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("AHPP_LARGE") != "1",
                    reason="large graph: about 3 minutes of host-side generation; set AHPP_LARGE=1")
def test_large_graph_properties(ahpp):
    g = synth.make_graph(**synth.LARGE)
    G = ahpp.Graph.from_arrays(g)
    try:
        info = G.info
        assert info["n_e"] == g.n_e and info["n_ea"] == g.n_ea
        qs = [int(x) for x in synth.draw_queries(g.n_u, 256)]
        eps = 1e-6
        alone, st, rc = G.query_dense(qs[0], eps)
        assert rc == 0 and st["mass_err"] < 1e-5 and alone.min() >= 0.0
        assert alone[qs[0]] >= ALPHA - TOL
        res = G.query_batch(qs, eps, 1000)       # 256-query batch, top-1,000
        assert all(r.rc == 0 and r.stats["mass_err"] < 1e-5 for r in res)
        top = res[0]
        assert top.nodes.shape[0] == 1000
        np.testing.assert_allclose(top.scores, alone[top.nodes], rtol=1e-5, atol=TOL)
        assert abs(res[0].stats["rounds"] - st["rounds"]) <= 1
        # Theorem 2 against the GPU's Algorithm 1 at T = 250
        pi_T, _, rc = G.power_iteration(qs[0], 250)
        assert rc == 0
        d = pi_T.astype(np.float64) - alone.astype(np.float64)
        assert d.min() >= -5e-7 and d.max() <= eps + 5e-7
        # serving on the large graph with the serving workload's request mix
        rng = np.random.default_rng(23)
        ns = 40
        sq = synth.draw_queries(g.n_u, ns, seed=29)
        se = np.exp(rng.uniform(np.log(1e-7), np.log(1e-4), ns))
        sk = rng.choice([10, 100, 1000], ns)
        srv = ahpp.Server(G, max_slots=32, rounds_per_step=8)
        try:
            tk = [srv.submit(int(sq[i]), float(se[i]), int(sk[i])) for i in range(ns)]
            sr = [srv.wait(t, int(k)) for t, k in zip(tk, sk)]
        finally:
            srv.stop()
        for i in (0, 17, 33, 39):
            assert sr[i].rc == 0 and sr[i].stats["mass_err"] < 1e-5
            one = G.query(int(sq[i]), float(se[i]), int(sk[i]))
            assert sr[i].stats["rounds"] == one.stats["rounds"]
            common = len(set(sr[i].nodes.tolist()) & set(one.nodes.tolist())) / int(sk[i])
            assert common >= 0.98
    finally:
        G.close()
