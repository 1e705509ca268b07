"""Parity at the full workload sizes, in the launch configuration bench.py times.

Every comparison below holds the parity bar: each score within 1e-6
absolute of the FP64 oracle push at every eps, within eps of exact AHPP
(Theorem 2) up to FP32 rounding, and top-k overlap >= 0.99 under the 2 eps
tie rule.  The oracle references (pushes, and exact AHPP by Algorithm 1 run
until (1 - alpha)^T <= 1e-10) are computed in spawned worker processes while
the GPU tests run (tests/oracle_jobs.py).

Medium (|U|=1M, |V|=500k, |E|=20M, |A|=10k x 20, bf16 attribute weights):
the single-query path and a 64-query batched launch element by element
against the oracle push; Theorem 2 against the oracle's exact AHPP; the
1,024-query launch bench.py times; the single-query workload's other eps;
the ablation arms of Exp-2 (APP, APP(S), APP(E), the printed switch rule)
against the oracle run with the same rule; and continuous batching with the
serving workload's request mix, every sampled request against the same
query alone and against the oracle.

Large, reduced (the large recipe with |U|, |V|, |E|, |A| scaled by 1/4:
1.25M / 1.25M / 50M edges, 12,500 x 30 attributes, Zipf(2.0)): one query
element by element against the oracle push and its exact AHPP; the
256-query batch with top-1,000.

Large (|U|=|V|=5M, |E|=200M, |A|=50k x 30): the oracle's exact push takes
too long for a test at this size, so the GPU's Algorithm 1 is pinned
element by element to the oracle's Algorithm 1 iterate at T = 12 and then
serves as the exact reference (T = 250, (1 - alpha)^250 < 1e-17) for
Theorem 2; the 256-query batch with top-1,000 and served requests are
compared with the query alone.
"""
import numpy as np
import pytest

import oracle
from oracle_jobs import Jobs, exact_T, pi_job, push_job
from paper_2512_11606_gb300 import synth
from parity_util import TOL, check_dense, check_topk

pytestmark = pytest.mark.gpu
ALPHA, BETA = 0.15, 0.35
FP32_SLACK = 5e-7          # pi_hat may exceed exact pi by FP32 rounding only
T_EXACT = exact_T(ALPHA)   # Algorithm 1 iterations with (1 - alpha)^T <= 1e-10

MED = synth.MEDIUM_BF16
MED_NU = MED["n_u"]
Q1024 = [int(x) for x in synth.draw_queries(MED_NU, 1024)]
Q_OTHER = int(synth.draw_queries(MED_NU, 2, seed=7)[1])
OTHER_EPS = (1e-5, 1e-7)
# the serving workload's request mix: eps log-uniform in [1e-7, 1e-4], k in {10, 100, 1000}
SERVE_N = 48
SERVE_Q = [int(x) for x in synth.draw_queries(MED_NU, SERVE_N, seed=61)]
_rng = np.random.default_rng(17)
SERVE_EPS = np.exp(_rng.uniform(np.log(1e-7), np.log(1e-4), SERVE_N))
SERVE_K = _rng.choice([10, 100, 1000], SERVE_N)
SERVE_CHECK = [0, 5, 23, 24, 30, 47]
# the ablation arms of Exp-2 at full size: (oracle algo, library algo name, switch rule)
ARMS = [("app", "AHPP_APP", 0), ("apps", "AHPP_APP_S", 0), ("asrp", "AHPP_ASRP", 2), ("asrp", "AHPP_ASRP", 1)]


@pytest.fixture(scope="module")
def ahpp():
    from paper_2512_11606_gb300 import build
    build.build()
    from paper_2512_11606_gb300 import ahpp as mod
    return mod


class Refs:
    """Oracle results by name, collected once from the background jobs."""

    def __init__(self, spec, named):
        self.names = [n for n, _ in named]
        self.jobs = Jobs(spec, [j for _, j in named])
        self.res = None

    def __getitem__(self, name):
        if self.res is None:
            self.res = dict(zip(self.names, self.jobs.get()))
        return self.res[name]


@pytest.fixture(scope="module")
def medium(ahpp):
    g = synth.make_graph(**MED)
    og = oracle.OracleGraph.from_arrays(g)
    lam, _ = og.lambda_estimate(ALPHA, BETA)
    named = [("q0", push_job(Q1024[0], 1e-6, lam)),
             ("exact0", pi_job(Q1024[0], T_EXACT)), ("exact63", pi_job(Q1024[63], T_EXACT))]
    named += [(f"other{e:g}", push_job(Q_OTHER, e, lam)) for e in OTHER_EPS]
    named += [(f"serve{i}", push_job(SERVE_Q[i], SERVE_EPS[i], lam)) for i in SERVE_CHECK]
    named += [(f"arm{a}{r}", push_job(Q_OTHER, 1e-6, lam, algo=a, switch_rule=r)) for a, _, r in ARMS]
    refs = Refs(MED, named)
    G = ahpp.Graph.from_arrays(g, lam=lam)
    yield dict(g=g, og=og, lam=lam, G=G, refs=refs)
    G.close()
    refs.jobs.cancel()


def test_medium_lambda_on_gpu_matches_oracle(ahpp, medium):
    G2 = ahpp.Graph.from_arrays(medium["g"])
    lam_gpu = G2.lam
    G2.close()
    assert lam_gpu >= medium["lam"] * (1 - 1e-6)
    assert abs(lam_gpu - medium["lam"]) / medium["lam"] <= 2e-4


def test_medium_single_and_batched_vs_oracle(medium):
    G, lam, refs = medium["G"], medium["lam"], medium["refs"]
    qs = Q1024[:64]
    eps = 1e-6
    alone, st, rc = G.query_dense(qs[0], eps)
    assert rc == 0
    dense, stats, rc = G.query_batch_dense(qs, eps)
    assert rc == 0
    for i in range(len(qs)):
        s = stats[i]
        assert s["status"] == 0 and s["mass_err"] < 1e-5
        assert dense[i].min() >= 0.0 and dense[i][qs[i]] >= ALPHA - TOL
        assert s["max_resid"] <= s["eps_f"] * (1 + 1e-6)
        assert s["eps_f"] <= eps / lam * (1 + 1e-6)
    pi_T, _, rc = G.power_iteration(qs[0], 250)
    assert rc == 0
    res = G.query_batch(Q1024, eps, 100)        # the launch bench.py times: 1,024 queries, top-100
    assert all(r.rc == 0 and r.stats["status"] == 0 for r in res)

    pi_ref, ref_stats = refs["q0"]
    check_dense(alone, pi_ref)
    assert abs(st["rounds"] - ref_stats["rounds"]) <= 1
    check_dense(dense[0], pi_ref)
    check_dense(dense[0], alone)
    # Theorem 2 against the oracle's exact AHPP: 0 <= pi - pi_hat <= eps
    for i, name in ((0, "exact0"), (63, "exact63")):
        exact, _ = refs[name]
        d = exact - dense[i].astype(np.float64)
        assert d.min() >= -FP32_SLACK and d.max() <= eps + FP32_SLACK, (d.min(), d.max())
    # the GPU's Algorithm 1 (the exact reference of the large test) against the oracle's
    check_dense(pi_T, refs["exact0"][0])
    check_topk(res[0].nodes, res[0].scores, pi_ref, 100, eps)
    for i in range(1, 64):
        check_topk(res[i].nodes, res[i].scores, dense[i], 100, eps)


@pytest.mark.parametrize("eps", OTHER_EPS)
def test_medium_single_query_other_eps(medium, eps):
    """The single-query workload's other error thresholds: every score within
    1e-6 of the oracle push, top-100 overlap with the oracle >= 0.99."""
    G, refs = medium["G"], medium["refs"]
    pi, st, rc = G.query_dense(Q_OTHER, eps)
    assert rc == 0 and st["status"] == 0
    top = G.query(Q_OTHER, eps, 100)
    pi_ref, ref_stats = refs[f"other{eps:g}"]
    check_dense(pi, pi_ref)
    assert abs(st["rounds"] - ref_stats["rounds"]) <= 1
    check_topk(top.nodes, top.scores, pi_ref, 100, eps)


@pytest.mark.parametrize("arm", ARMS, ids=["app", "apps", "app_e", "asrp_printed_switch"])
def test_medium_ablation_arms_vs_oracle(ahpp, medium, arm):
    """The ablation arms of Exp-2 at the medium size: APP, APP(S), APP(E)
    (ASRP never switching) and ASRP with the switch budget as printed, each
    through the single-query and the batched launch, every score within 1e-6
    of the oracle run with the same rule, rounds within one of the oracle's
    (three for APP, whose stop test is per node)."""
    oalgo, lib_algo, rule = arm
    G = ahpp.Graph.from_arrays(medium["g"], lam=medium["lam"], algo=getattr(ahpp, lib_algo),
                               switch_rule=rule)
    try:
        pi, st, rc = G.query_dense(Q_OTHER, 1e-6)
        dense, stats, rc_b = G.query_batch_dense([Q_OTHER] + Q1024[:7], 1e-6)
    finally:
        G.close()
    assert rc == 0 and rc_b == 0 and st["status"] == 0 and stats[0]["status"] == 0
    pi_ref, ref_stats = medium["refs"][f"arm{oalgo}{rule}"]
    check_dense(pi, pi_ref)
    check_dense(dense[0], pi_ref)
    # APP stops once every residue is at most r_max (|N(u)| + |A(u)|), about
    # 1e-12 here: FP32 residues that close to their thresholds (about 1e-7
    # relative from the oracle's FP64) can keep a node pushing a round or two
    # longer; the other arms stop on a test that FP32 rounding does not reach
    # (eps / lambda, about 2.4e-10, or APP(S)'s synchronous sweep of every
    # residue) and agree within one round
    tol = 3 if oalgo == "app" else 1
    assert abs(st["rounds"] - ref_stats["rounds"]) <= tol
    assert abs(stats[0]["rounds"] - ref_stats["rounds"]) <= tol


def test_medium_served_mix_equals_alone(ahpp, medium):
    """Continuous batching at full size with the serving workload's request
    mix: requests admitted while others run; every sampled request equals the
    same query alone (its dense vector) and the oracle push, within 1e-6."""
    G, refs = medium["G"], medium["refs"]
    srv = ahpp.Server(G, max_slots=32, rounds_per_step=8)
    try:
        tickets = [srv.submit(SERVE_Q[i], float(SERVE_EPS[i]), int(SERVE_K[i])) for i in range(24)]
        first = srv.wait(tickets[0], int(SERVE_K[0]))
        tickets += [srv.submit(SERVE_Q[i], float(SERVE_EPS[i]), int(SERVE_K[i]))
                    for i in range(24, SERVE_N)]
        results = [first] + [srv.wait(t, int(k)) for t, k in zip(tickets[1:], SERVE_K[1:])]
        info = srv.info()
        assert info["completed"] == SERVE_N and info["steps"] > 1
    finally:
        srv.stop()
    for i in SERVE_CHECK:
        r, e, k = results[i], float(SERVE_EPS[i]), int(SERVE_K[i])
        assert r.rc == 0 and r.stats["status"] == 0 and r.stats["mass_err"] < 1e-5
        alone, st, rc = G.query_dense(SERVE_Q[i], e)
        assert rc == 0 and r.stats["rounds"] == st["rounds"]
        check_topk(r.nodes, r.scores, alone, k, e)
        pi_ref, ref_stats = refs[f"serve{i}"]
        check_dense(alone, pi_ref)
        check_topk(r.nodes, r.scores, pi_ref, k, e)
        assert abs(r.stats["rounds"] - ref_stats["rounds"]) <= 1


def test_large_reduced_vs_oracle(ahpp):
    """The large recipe at 1/4 scale: one query element by element against
    the oracle push (the oracle is given the GPU's Theorem 3 estimate, whose
    agreement with the oracle's own is tested on the medium graph) and
    against exact AHPP; the 256-query batch with top-1,000."""
    spec = synth.scaled(synth.LARGE, 0.25)
    g = synth.make_graph(**spec)
    G = ahpp.Graph.from_arrays(g)
    try:
        lam = G.lam
        qs = [int(x) for x in synth.draw_queries(g.n_u, 256)]
        eps = 1e-6
        refs = Refs(spec, [("push", push_job(qs[0], eps, lam)), ("exact", pi_job(qs[0], T_EXACT))])
        alone, st, rc = G.query_dense(qs[0], eps)
        assert rc == 0 and st["mass_err"] < 1e-5
        res = G.query_batch(qs, eps, 1000)
        assert all(r.rc == 0 and r.stats["mass_err"] < 1e-5 for r in res)
        dense, bst, rc = G.query_batch_dense(qs[:32], eps)
        assert rc == 0
        pi_ref, ref_stats = refs["push"]
        check_dense(alone, pi_ref)
        check_dense(dense[0], pi_ref)
        assert abs(st["rounds"] - ref_stats["rounds"]) <= 1
        exact, _ = refs["exact"]
        d = exact - alone.astype(np.float64)
        assert d.min() >= -FP32_SLACK and d.max() <= eps + FP32_SLACK, (d.min(), d.max())
        check_topk(res[0].nodes, res[0].scores, pi_ref, 1000, eps)
        for i in (1, 17, 31):
            check_topk(res[i].nodes, res[i].scores, dense[i], 1000, eps)
    finally:
        G.close()


def test_large_graph(ahpp):
    """The large workload (5M / 5M / 200M edges, 50k x 30 attributes): the
    GPU's Algorithm 1 against the oracle's iterate at T = 12 (element by
    element), Theorem 2 against the GPU's Algorithm 1 at T = 250, the
    256-query batch with top-1,000 against the queries alone, and served
    requests of the serving workload's mix against the queries alone."""
    spec = synth.LARGE
    T_PIN = 12
    qs = [int(x) for x in synth.draw_queries(spec["n_u"], 256)]
    refs = Refs(spec, [("pi12", pi_job(qs[0], T_PIN))])     # the worker builds its own copy
    g = synth.make_graph(**spec)
    G = ahpp.Graph.from_arrays(g)
    try:
        info = G.info
        assert info["n_e"] == g.n_e and info["n_ea"] == g.n_ea
        eps = 1e-6
        alone, st, rc = G.query_dense(qs[0], eps)
        assert rc == 0 and st["mass_err"] < 1e-5 and alone.min() >= 0.0
        assert alone[qs[0]] >= ALPHA - TOL
        res = G.query_batch(qs, eps, 1000)       # 256-query batch, top-1,000
        assert all(r.rc == 0 and r.stats["mass_err"] < 1e-5 for r in res)
        check_topk(res[0].nodes, res[0].scores, alone, 1000, eps)
        assert abs(res[0].stats["rounds"] - st["rounds"]) <= 1
        for i in (101, 255):
            one, _, _ = G.query_dense(qs[i], eps)
            check_topk(res[i].nodes, res[i].scores, one, 1000, eps)
        pi_T, _, rc = G.power_iteration(qs[0], 250)
        assert rc == 0
        d = pi_T.astype(np.float64) - alone.astype(np.float64)
        assert d.min() >= -FP32_SLACK and d.max() <= eps + FP32_SLACK, (d.min(), d.max())
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
            one, ost, _ = G.query_dense(int(sq[i]), float(se[i]))
            assert sr[i].stats["rounds"] == ost["rounds"]
            check_topk(sr[i].nodes, sr[i].scores, one, int(sk[i]), float(se[i]))
        pi12, _, rc = G.power_iteration(qs[0], T_PIN)
        assert rc == 0
        check_dense(pi12, refs["pi12"][0])
    finally:
        G.close()
        refs.jobs.cancel()
