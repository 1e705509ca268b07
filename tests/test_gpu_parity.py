"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance: every reserve within 1e-6 absolute of the oracle's push at every
eps (the GPU follows the oracle's trajectory: the round counts are compared
too, and FP32 rounding is the only expected difference), and within eps of
exact AHPP (Theorem 2) up to FP32 rounding (1e-7).
"""
import numpy as np
import pytest

import oracle
from paper_2512_11606_gb300 import synth
from parity_util import check_topk

pytestmark = pytest.mark.gpu

ALPHA, BETA = 0.15, 0.35
TOL = 1e-6          # |gpu - oracle push|
FP32_SLACK = 1e-7   # pi_hat may exceed exact pi by FP32 rounding only


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
    _, _, P = oracle.dense_matrices_of(g, BETA)
    Pi = oracle.pi_matrix(P, ALPHA)
    G = ahpp.Graph.from_arrays(g, lam=lam, attr_bf16=0)
    qs = [int(x) for x in synth.draw_queries(g.n_u, 4)]
    yield dict(g=g, og=og, lam=lam, Pi=Pi, G=G, qs=qs)
    G.close()


def check_dense(pi_gpu, ref_pi, exact, eps):
    pi_gpu = pi_gpu.astype(np.float64)
    d = np.abs(pi_gpu - ref_pi).max()
    assert d <= TOL, d
    err = exact - pi_gpu
    assert err.min() >= -FP32_SLACK, err.min()
    assert err.max() <= eps + FP32_SLACK, (err.max(), eps)
    return d


def test_lambda_estimate_matches_oracle(ahpp, tiny):
    G2 = ahpp.Graph.from_arrays(tiny["g"], attr_bf16=0)
    lam_gpu, lam = G2.lam, tiny["lam"]
    G2.close()
    assert lam_gpu >= lam * (1 - 1e-6)
    assert abs(lam_gpu - lam) / lam <= 2e-4
    colsum = tiny["Pi"].sum(axis=0).max()
    assert lam_gpu >= colsum           # Theorem 3 holds for the GPU estimate too


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_asrp_dense_parity(tiny, eps):
    G, og, lam = tiny["G"], tiny["og"], tiny["lam"]
    for q in tiny["qs"]:
        pi_gpu, st, rc = G.query_dense(q, eps)
        assert rc == 0 and st["status"] == 0
        ref = og.push("asrp", ALPHA, BETA, q, eps, lam=lam)
        check_dense(pi_gpu, ref.pi, tiny["Pi"][q], eps)
        assert abs(st["rounds"] - ref.stats["rounds"]) <= 1
        assert st["mass_err"] < 1e-5
        assert pi_gpu.min() >= 0


def test_asrp_trajectory_and_switch(tiny):
    G, og, lam = tiny["G"], tiny["og"], tiny["lam"]
    q = tiny["qs"][0]
    _, st, _ = G.query_dense(q, 1e-6)
    ref = og.push("asrp", ALPHA, BETA, q, 1e-6, lam=lam)
    assert st["rounds"] == ref.stats["rounds"]
    assert st["switch_round"] == ref.stats["switch_round"]
    assert st["n_p"] == ref.stats["n_p"]
    assert st["pushes"] == ref.stats["pushes"]


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_app_dense_parity(ahpp, tiny, eps):
    G = ahpp.Graph.from_arrays(tiny["g"], algo=ahpp.AHPP_APP, attr_bf16=0)
    try:
        for q in tiny["qs"][:2]:
            pi_gpu, st, rc = G.query_dense(q, eps)
            assert rc == 0
            ref = tiny["og"].push("app", ALPHA, BETA, q, eps)
            check_dense(pi_gpu, ref.pi, tiny["Pi"][q], eps)
            assert abs(st["rounds"] - ref.stats["rounds"]) <= 1
    finally:
        G.close()


@pytest.mark.parametrize("vw", [1, 4, 8, 16, 32])
def test_short_row_lane_widths_match_oracle(ahpp, tiny, vw):
    """The single-query kernel walks short rows with up to vw lanes each (the
    default 2 is covered by every other test): the same result for each."""
    G = ahpp.Graph.from_arrays(tiny["g"], lam=tiny["lam"], attr_bf16=0, single_vec_width=vw)
    try:
        assert G.info["single_vec_width"] == vw
        for q in tiny["qs"][:2]:
            pi, st, rc = G.query_dense(q, 1e-6)
            assert rc == 0
            ref = tiny["og"].push("asrp", ALPHA, BETA, q, 1e-6, lam=tiny["lam"])
            check_dense(pi, ref.pi, tiny["Pi"][q], 1e-6)
            assert abs(st["rounds"] - ref.stats["rounds"]) <= 1
    finally:
        G.close()


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_apps_dense_parity(ahpp, tiny, eps):
    """APP(S) (APP's thresholds with the synchronous switch, Exp-2's ablation
    arm): the single-query kernel follows the oracle's trajectory (rounds,
    switch round) and every reserve is within 1e-6 of the oracle push."""
    G = ahpp.Graph.from_arrays(tiny["g"], algo=ahpp.AHPP_APP_S, attr_bf16=0)
    try:
        for q in tiny["qs"][:3]:
            pi_gpu, st, rc = G.query_dense(q, eps)
            assert rc == 0 and st["status"] == 0
            ref = tiny["og"].push("apps", ALPHA, BETA, q, eps)
            check_dense(pi_gpu, ref.pi, tiny["Pi"][q], eps)
            assert abs(st["rounds"] - ref.stats["rounds"]) <= 1
            assert abs(st["switch_round"] - ref.stats["switch_round"]) <= 1
            assert ref.stats["switch_round"] > 0 or eps > 1e-5
    finally:
        G.close()


def topk_overlap(nodes, ref_scores, k, eps):
    """Overlap with the oracle's top-k; nodes whose oracle score lies within
    2 eps of the k-th score are interchangeable (ties of the approximation)."""
    order = np.lexsort((np.arange(ref_scores.shape[0]), -ref_scores))
    kth = ref_scores[order[k - 1]]
    sure = set(order[:k][ref_scores[order[:k]] > kth + 2 * eps].tolist())
    ok = set(np.nonzero(ref_scores >= kth - 2 * eps)[0].tolist())
    got = set(int(x) for x in nodes)
    assert sure <= got, sorted(sure - got)[:10]
    return len(got & ok) / k


@pytest.mark.parametrize("k", [1, 50, 500])
def test_topk_single(tiny, k):
    G, og, lam = tiny["G"], tiny["og"], tiny["lam"]
    q, eps = tiny["qs"][1], 1e-6
    res = G.query(q, eps, k)
    dense, _, _ = G.query_dense(q, eps)
    assert res.nodes.shape[0] == k
    # order: score descending, then id ascending
    key = np.lexsort((res.nodes, -res.scores))
    np.testing.assert_array_equal(key, np.arange(k))
    # the two calls are separate runs whose FP32 atomic sums may differ in the
    # last bits; scores agree with the dense vector to FP32 rounding
    np.testing.assert_allclose(res.scores, dense[res.nodes], rtol=1e-6, atol=1e-9)
    ref = og.push("asrp", ALPHA, BETA, q, eps, lam=lam)
    assert topk_overlap(res.nodes, ref.pi, k, eps) >= 0.99
    # the top-k of the GPU's own dense vector, up to ties within FP32 rounding
    assert topk_overlap(res.nodes, dense.astype(np.float64), k, 1e-8) >= 0.99


def test_topk_k_larger_than_U(tiny):
    G = tiny["G"]
    res = G.query(tiny["qs"][0], 1e-4, 4096)
    assert res.nodes.shape[0] == tiny["g"].n_u
    assert sorted(res.nodes.tolist()) == list(range(tiny["g"].n_u))


def test_batch_alone_vs_mix(tiny):
    """A query's result is the same alone and inside a batch (3 tiles, ragged)."""
    G = tiny["G"]
    qs = [int(x) for x in synth.draw_queries(tiny["g"].n_u, 70, seed=5)]
    qs[10] = qs[11]                      # duplicate sources in one tile
    eps = np.where(np.arange(70) % 3 == 0, 1e-4, 1e-6)
    dense, stats, rc = G.query_batch_dense(qs, eps)
    assert rc == 0
    for i in [0, 1, 10, 11, 33, 64, 69]:
        alone, st, _ = G.query_dense(qs[i], eps[i])
        assert np.abs(dense[i] - alone).max() <= TOL
        assert stats[i]["rounds"] == st["rounds"]
        ref = tiny["og"].push("asrp", ALPHA, BETA, qs[i], eps[i], lam=tiny["lam"])
        check_dense(dense[i], ref.pi, tiny["Pi"][qs[i]], eps[i])


def test_narrow_tiles_match_oracle(ahpp, tiny):
    """Tiles of 16 queries (the batched kernel's other width): a ragged batch
    of three tiles with duplicate sources and mixed eps, element by element
    against the oracle and the same queries in tiles of 32; top-k too."""
    g, og, lam = tiny["g"], tiny["og"], tiny["lam"]
    G = ahpp.Graph.from_arrays(g, lam=lam, attr_bf16=0, batch_tile=16)
    try:
        assert G.info["batch_tile"] == 16
        qs = [int(x) for x in synth.draw_queries(g.n_u, 37, seed=8)]
        qs[3] = qs[4]
        eps = np.where(np.arange(37) % 3 == 0, 1e-4, 1e-6)
        dense, stats, rc = G.query_batch_dense(qs, eps)
        assert rc == 0
        wide, wstats, _ = tiny["G"].query_batch_dense(qs, eps)
        assert np.abs(dense - wide).max() <= TOL
        assert [s["rounds"] for s in stats] == [s["rounds"] for s in wstats]
        for i in (0, 3, 4, 15, 16, 36):
            ref = og.push("asrp", ALPHA, BETA, qs[i], float(eps[i]), lam=lam)
            check_dense(dense[i], ref.pi, tiny["Pi"][qs[i]], float(eps[i]))
        res = G.query_batch(qs, eps, 30)
        for i in (0, 16, 36):
            check_topk(res[i].nodes, res[i].scores, dense[i], 30, float(eps[i]))
    finally:
        G.close()


def test_batch_topk_matches_single(tiny):
    G = tiny["G"]
    qs = [int(x) for x in synth.draw_queries(tiny["g"].n_u, 40, seed=6)]
    ks = [50 if i % 2 else 7 for i in range(40)]
    res = G.query_batch(qs, 1e-6, ks)
    for i in [0, 1, 31, 32, 39]:
        alone, _, _ = G.query_dense(qs[i], 1e-6)
        check_topk(res[i].nodes, res[i].scores, alone, ks[i], 1e-6)
        one = G.query(qs[i], 1e-6, ks[i])
        check_topk(one.nodes, one.scores, alone, ks[i], 1e-6)


def test_invalid_arguments(ahpp, tiny):
    G = tiny["G"]
    with pytest.raises(ahpp.AhppError) as e:
        G.query(tiny["g"].n_u, 1e-6, 10)
    assert e.value.code == ahpp.AHPP_EINVAL
    with pytest.raises(ahpp.AhppError):
        G.query(0, 0.0, 10)
    with pytest.raises(ahpp.AhppError):
        G.query(0, 1e-6, ahpp.AHPP_MAX_K + 1)
    g = tiny["g"]
    bad = synth.GraphArrays(g.n_u, g.n_v, g.n_a, g.e_u, g.e_v, -g.e_w, g.ea_u, g.ea_a, g.ea_w)
    with pytest.raises(ahpp.AhppError):
        ahpp.Graph.from_arrays(bad)
    with pytest.raises(ahpp.AhppError):
        ahpp.Graph.from_arrays(g, alpha=1.5)


def small_graph(seed, n_u=300, n_v=200, n_e=1500, n_a=40, drop_attr=0.2, isolated_v=5):
    rng = np.random.default_rng(seed)
    e_u = rng.integers(0, n_u, n_e).astype(np.uint32)
    e_v = rng.integers(0, n_v - isolated_v, n_e).astype(np.uint32)   # last V nodes isolated
    e_w = rng.uniform(0.5, 1.5, n_e).astype(np.float32)
    keep = rng.random(n_u) > drop_attr
    au = np.repeat(np.nonzero(keep)[0], 3).astype(np.uint32)
    aa = rng.integers(0, n_a, au.shape[0]).astype(np.uint32)           # duplicates possible
    aw = rng.uniform(0.1, 1.0, au.shape[0]).astype(np.float32)
    return synth.GraphArrays(n_u, n_v, n_a, e_u, e_v, e_w, au, aa, aw)


@pytest.mark.parametrize("seed", [0, 1])
def test_dangling_duplicates_isolated(ahpp, seed):
    """Duplicate pairs, U nodes without attributes or edges, isolated V nodes."""
    g = small_graph(seed)
    og = oracle.OracleGraph.from_arrays(g)
    lam, _ = og.lambda_estimate(ALPHA, BETA)
    _, _, P = oracle.dense_matrices_of(g, BETA)
    G = ahpp.Graph.from_arrays(g, lam=lam, attr_bf16=0)
    try:
        assert G.info["n_e"] == og.n_e and G.info["n_ea"] == og.n_ea
        for q in [0, 7, 150]:
            pi_gpu, st, rc = G.query_dense(q, 1e-7)
            ref = og.push("asrp", ALPHA, BETA, q, 1e-7, lam=lam)
            check_dense(pi_gpu, ref.pi, oracle.exact_dense(P, ALPHA, q), 1e-7)
    finally:
        G.close()


def test_closed_form_hub(ahpp):
    n = 17
    u = np.arange(n, dtype=np.uint32)
    z = np.zeros(n, dtype=np.uint32)
    one = np.ones(n, dtype=np.float32)
    G = ahpp.Graph(n, 1, 1, u, z, one, u, z, one)
    try:
        pi, st, rc = G.query_dense(3, 1e-9)
        want = np.full(n, (1 - ALPHA) / n)
        want[3] += ALPHA
        d = want - pi.astype(np.float64)
        assert d.min() >= -FP32_SLACK and d.max() <= 1e-9 + FP32_SLACK
    finally:
        G.close()


@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_beta_extremes(ahpp, tiny, beta):
    g, og = tiny["g"], tiny["og"]
    lam, _ = og.lambda_estimate(ALPHA, beta)
    _, _, P = oracle.dense_matrices_of(g, beta)
    G = ahpp.Graph.from_arrays(g, beta=beta, lam=lam, attr_bf16=0)
    try:
        q = tiny["qs"][2]
        pi, _, rc = G.query_dense(q, 1e-6)
        ref = og.push("asrp", ALPHA, beta, q, 1e-6, lam=lam)
        check_dense(pi, ref.pi, oracle.exact_dense(P, ALPHA, q), 1e-6)
    finally:
        G.close()


def test_bf16_attribute_weights(ahpp):
    """bfloat16 storage: the oracle gets the same bf16-representable weights."""
    g = synth.make_graph(**dict(synth.TINY, bf16=True))
    og = oracle.OracleGraph.from_arrays(g)
    lam, _ = og.lambda_estimate(ALPHA, BETA)
    _, _, P = oracle.dense_matrices_of(g, BETA)
    G = ahpp.Graph.from_arrays(g, lam=lam, attr_bf16=1)
    try:
        for q in [int(x) for x in synth.draw_queries(g.n_u, 2, seed=9)]:
            pi, _, _ = G.query_dense(q, 1e-6)
            ref = og.push("asrp", ALPHA, BETA, q, 1e-6, lam=lam)
            check_dense(pi, ref.pi, oracle.exact_dense(P, ALPHA, q), 1e-6)
    finally:
        G.close()


def test_kahan_off_still_within_tolerance(ahpp, tiny):
    G = ahpp.Graph.from_arrays(tiny["g"], lam=tiny["lam"], attr_bf16=0, kahan=0)
    try:
        q = tiny["qs"][3]
        pi, _, _ = G.query_dense(q, 1e-6)
        ref = tiny["og"].push("asrp", ALPHA, BETA, q, 1e-6, lam=tiny["lam"])
        check_dense(pi, ref.pi, tiny["Pi"][q], 1e-6)
    finally:
        G.close()


def test_round_cap_reports_not_converged(ahpp, tiny):
    G = ahpp.Graph.from_arrays(tiny["g"], lam=tiny["lam"], attr_bf16=0, max_rounds=3)
    try:
        pi, st, rc = G.query_dense(tiny["qs"][0], 1e-6)
        assert rc == ahpp.AHPP_ENOTCONVERGED and st["rounds"] == 3 and st["status"] == 1
        ref = tiny["og"].push("asrp", ALPHA, BETA, tiny["qs"][0], 1e-6, lam=tiny["lam"],
                              max_rounds=3)
        assert np.abs(pi - ref.pi).max() <= TOL
    finally:
        G.close()


@pytest.mark.parametrize("T", [1, 2, 10, 60])
def test_power_iteration_matches_oracle(tiny, T):
    """Algorithm 1 on the GPU: the oracle's iterate after T steps, and within
    (1 - alpha)^T of exact AHPP."""
    G, og = tiny["G"], tiny["og"]
    for q in tiny["qs"][:2]:
        pi_gpu, st, rc = G.power_iteration(q, T)
        assert rc == 0 and st["rounds"] == T
        ref = og.power_iteration(ALPHA, BETA, q, T)
        assert np.abs(pi_gpu.astype(np.float64) - ref).max() <= TOL
        assert np.abs(tiny["Pi"][q] - pi_gpu).max() <= (1 - ALPHA) ** T + TOL
        assert abs(pi_gpu.astype(np.float64).sum() - 1.0) <= 1e-5


def test_power_iteration_one_step_closed_form(tiny):
    """T = 1: alpha e_q + (1 - alpha) e_q P, with P from its definition."""
    G, g = tiny["G"], tiny["g"]
    _, _, P = oracle.dense_matrices_of(g, BETA)
    q = tiny["qs"][1]
    pi_gpu, _, _ = G.power_iteration(q, 1)
    want = (1 - ALPHA) * P[q]
    want[q] += ALPHA
    assert np.abs(pi_gpu - want).max() <= 1e-7


def test_power_iteration_invalid(ahpp, tiny):
    G = tiny["G"]
    for q, T in [(0, 0), (tiny["g"].n_u, 5), (0, 100001)]:
        with pytest.raises(ahpp.AhppError) as e:
            G.power_iteration(q, T)
        assert e.value.code == ahpp.AHPP_EINVAL


def test_source_below_threshold_pushes_nothing(ahpp, tiny):
    """The degenerate case of Algorithms 3 and 4: with eps / lambda above the
    source's unit residue no node is ever selected, so the result is the
    zero vector after 0 rounds (the oracle agrees), and its top-k are the k
    smallest caller ids at score 0 (score descending, id ascending).  Single
    query, a batched launch whose other lane is an ordinary query, and the
    server."""
    G, og, lam, q, q2 = tiny["G"], tiny["og"], tiny["lam"], tiny["qs"][0], tiny["qs"][1]
    big = 2.0 * lam                                # eps_f = 2 > r(q) = 1
    ref = og.push("asrp", ALPHA, BETA, q, big, lam=lam)
    assert ref.stats["rounds"] == 0 and not ref.pi.any()
    pi, st, rc = G.query_dense(q, big)
    assert rc == 0 and st["status"] == 0 and st["rounds"] == 0 and not pi.any()
    top = G.query(q, big, 5)
    assert top.nodes.tolist() == [0, 1, 2, 3, 4] and not top.scores.any()
    dense, stats, rc = G.query_batch_dense([q, q2], [big, 1e-6])
    assert rc == 0 and stats[0]["rounds"] == 0 and not dense[0].any()
    ref2 = og.push("asrp", ALPHA, BETA, q2, 1e-6, lam=lam)
    assert np.abs(dense[1].astype(np.float64) - ref2.pi).max() <= TOL
    res = G.query_batch([q, q2], [big, 1e-6], 5)
    assert res[0].nodes.tolist() == [0, 1, 2, 3, 4] and not res[0].scores.any()
    srv = ahpp.Server(G, max_slots=32, rounds_per_step=2)
    try:
        t = [srv.submit(q, big, 5), srv.submit(q2, 1e-6, 5)]
        r0, r1 = srv.wait(t[0], 5), srv.wait(t[1], 5)
    finally:
        srv.stop()
    assert r0.stats["rounds"] == 0 and r0.nodes.tolist() == [0, 1, 2, 3, 4] and not r0.scores.any()
    assert r1.nodes.tolist() == res[1].nodes.tolist()
