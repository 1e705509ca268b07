"""The remaining public paths of the C ABI against the host paths and the oracle.

Device-resident calls (the launch bench.py times), the ASRP switch rules,
concurrent tile groups and the autotuner, APP in the batched kernel, the
batch edge cases (empty batch, k clamped to |U|), and the device-side
failure detection (a bounded wait that gives up and reports it).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2512_11606_gb300 import synth
from parity_util import check_topk

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


def stats_of(ahpp, raw):
    """Decode a [n, sizeof(ahpp_stats)] byte tensor into dicts."""
    n = raw.shape[0]
    buf = (ahpp.Stats * n).from_buffer_copy(raw.cpu().numpy().tobytes())
    return [buf[i].as_dict() for i in range(n)]


def test_device_batch_matches_host(ahpp, tiny):
    torch = pytest.importorskip("torch")
    G, g = tiny["G"], tiny["g"]
    n, kmax = 45, 50
    qs = synth.draw_queries(g.n_u, n, seed=71).astype(np.int64)
    ks = np.where(np.arange(n) % 2 == 0, 50, 13)
    dev = torch.device("cuda", 0)
    q_t = torch.tensor(qs, dtype=torch.int32, device=dev)
    eps_t = torch.full((n,), 1e-6, dtype=torch.float64, device=dev)
    k_t = torch.tensor(ks, dtype=torch.int32, device=dev)
    nodes_t = torch.full((n, kmax), -1, dtype=torch.int32, device=dev)
    scores_t = torch.zeros((n, kmax), dtype=torch.float32, device=dev)
    n_t = torch.zeros(n, dtype=torch.int32, device=dev)
    st_t = torch.zeros((n, ahpp.STATS_BYTES), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    rc = G.query_batch_device(q_t, eps_t, k_t, kmax, nodes_t, scores_t, n_t, st_t, stream)
    stream.synchronize()
    assert rc == 0
    host = G.query_batch([int(x) for x in qs], 1e-6, ks.astype(np.uint32))
    dense, _, _ = G.query_batch_dense([int(x) for x in qs], 1e-6)
    dst = stats_of(ahpp, st_t)
    cnt = n_t.cpu().numpy()
    nodes = nodes_t.cpu().numpy()
    scores = scores_t.cpu().numpy()
    for i in range(n):
        assert cnt[i] == ks[i]
        h = host[i]
        check_topk(nodes[i, :cnt[i]], scores[i, :cnt[i]], dense[i], ks[i], 1e-6)
        check_topk(h.nodes, h.scores, dense[i], ks[i], 1e-6)
        assert dst[i]["rounds"] == h.stats["rounds"] and dst[i]["status"] == 0
        assert dst[i]["mass_err"] < 1e-5


def test_device_single_matches_host(ahpp, tiny):
    torch = pytest.importorskip("torch")
    G, g = tiny["G"], tiny["g"]
    dev = torch.device("cuda", 0)
    k = 40
    nodes_t = torch.zeros(k, dtype=torch.int32, device=dev)
    scores_t = torch.zeros(k, dtype=torch.float32, device=dev)
    n_t = torch.zeros(1, dtype=torch.int32, device=dev)
    st_t = torch.zeros((1, ahpp.STATS_BYTES), dtype=torch.uint8, device=dev)
    for q in synth.draw_queries(g.n_u, 3, seed=72):
        rc = G.query_device(int(q), 1e-6, k, nodes_t, scores_t, n_t, st_t, None)
        torch.cuda.synchronize()
        assert rc == 0
        h = G.query(int(q), 1e-6, k)
        assert int(n_t.item()) == k
        np.testing.assert_allclose(scores_t.cpu().numpy(), h.scores, atol=TOL)
        assert stats_of(ahpp, st_t)[0]["rounds"] == h.stats["rounds"]


@pytest.mark.parametrize("rule", [1, 2])
def test_switch_rules_match_oracle(ahpp, tiny, rule):
    """switch_rule 1 (the printed formula) and 2 (never switch): single and
    batched results follow the oracle run with the same rule."""
    g, og, lam = tiny["g"], tiny["og"], tiny["lam"]
    G = ahpp.Graph.from_arrays(g, lam=lam, attr_bf16=0, switch_rule=rule)
    try:
        qs = [int(x) for x in synth.draw_queries(g.n_u, 3, seed=73)]
        dense, stats, rc = G.query_batch_dense(qs, 1e-6)
        assert rc == 0
        for i, q in enumerate(qs):
            ref = og.push("asrp", ALPHA, BETA, q, 1e-6, lam=lam, switch_rule=rule)
            one, st, rc1 = G.query_dense(q, 1e-6)
            assert rc1 == 0
            assert np.abs(one.astype(np.float64) - ref.pi).max() <= TOL
            assert np.abs(dense[i].astype(np.float64) - ref.pi).max() <= TOL
            assert abs(st["rounds"] - ref.stats["rounds"]) <= 1
            if rule == 2:
                assert st["switch_round"] == 0 and ref.stats["switch_round"] == 0
    finally:
        G.close()


@pytest.mark.parametrize("groups", [2, 4])
def test_concurrent_tile_groups_same_results(ahpp, tiny, groups):
    g, lam = tiny["g"], tiny["lam"]
    qs = [int(x) for x in synth.draw_queries(g.n_u, 150, seed=74)]
    base, st0, _ = tiny["G"].query_batch_dense(qs, 1e-6)
    G = ahpp.Graph.from_arrays(g, lam=lam, attr_bf16=0, batch_groups=groups)
    try:
        assert G.info["batch_groups"] == groups
        dense, st, rc = G.query_batch_dense(qs, 1e-6)
        assert rc == 0
        assert np.abs(dense - base).max() <= TOL
        assert [s["rounds"] for s in st] == [s["rounds"] for s in st0]
    finally:
        G.close()


def test_autotune_keeps_results(ahpp, tiny):
    """The autotuner picks a shape among its candidates (tile groups, long-row
    chunk, push/pull cut of the single-query path) and the results under the
    tuned shape stay within 1e-6 of the oracle push, batched and single."""
    g, og, lam = tiny["g"], tiny["og"], tiny["lam"]
    G = ahpp.Graph.from_arrays(g, lam=lam, attr_bf16=0)
    try:
        qs = [int(x) for x in synth.draw_queries(g.n_u, 64, seed=75)]
        before, _, _ = G.query_batch_dense(qs, 1e-6)
        assert G.info["batch_chunk"] == 256 and G.info["single_dense_div"] == 32
        info = G.autotune(qs, 1e-6)
        assert info["batch_groups"] in (1, 2, 4) and info["batch_tile"] in (16, 32)
        assert info["batch_chunk"] in (128, 256, 512)
        assert info["single_dense_div"] in (8, 16, 32, 64, 128)
        assert info["single_vec_width"] in (1, 2, 8, 32)
        rep = G.autotune_report()
        assert "batch_groups=4" in rep and "single_dense_div=128" in rep and all(v > 0 for v in rep.values())
        after, _, rc = G.query_batch_dense(qs, 1e-6)
        assert rc == 0 and np.abs(after - before).max() <= TOL
        for i in (0, 33, 63):
            ref = og.push("asrp", ALPHA, BETA, qs[i], 1e-6, lam=lam)
            assert np.abs(after[i].astype(np.float64) - ref.pi).max() <= TOL
            one, _, rc1 = G.query_dense(qs[i], 1e-6)
            assert rc1 == 0 and np.abs(one.astype(np.float64) - ref.pi).max() <= TOL
    finally:
        G.close()


@pytest.mark.parametrize("chunk", [128, 512])
def test_every_chunk_choice_matches_oracle(ahpp, tiny, chunk):
    """Each long-row chunk size the autotuner may pick (set here through the
    configuration) gives the oracle's result in the batched kernel."""
    g, og, lam = tiny["g"], tiny["og"], tiny["lam"]
    G = ahpp.Graph.from_arrays(g, lam=lam, attr_bf16=0, batch_chunk=chunk)
    try:
        assert G.info["batch_chunk"] == chunk
        qs = [int(x) for x in synth.draw_queries(g.n_u, 40, seed=77)]
        dense, _, rc = G.query_batch_dense(qs, 1e-6)
        assert rc == 0
        for i in (0, 17, 39):
            ref = og.push("asrp", ALPHA, BETA, qs[i], 1e-6, lam=lam)
            assert np.abs(dense[i].astype(np.float64) - ref.pi).max() <= TOL
    finally:
        G.close()


def test_batched_app_matches_oracle(ahpp, tiny):
    g, og = tiny["g"], tiny["og"]
    G = ahpp.Graph.from_arrays(g, algo=ahpp.AHPP_APP, attr_bf16=0)
    try:
        qs = [int(x) for x in synth.draw_queries(g.n_u, 35, seed=76)]
        eps = np.where(np.arange(35) % 2 == 0, 1e-6, 1e-4)
        dense, stats, rc = G.query_batch_dense(qs, eps)
        assert rc == 0
        for i in [0, 1, 17, 33, 34]:
            ref = og.push("app", ALPHA, BETA, qs[i], float(eps[i]))
            assert np.abs(dense[i].astype(np.float64) - ref.pi).max() <= TOL
            assert abs(stats[i]["rounds"] - ref.stats["rounds"]) <= 1
            one, _, _ = G.query_dense(qs[i], float(eps[i]))
            assert np.abs(one - dense[i]).max() <= TOL
    finally:
        G.close()


def test_batched_and_served_apps_match_oracle(ahpp, tiny):
    """APP(S) in the batched kernel (per-lane thresholds, switch and stopping
    test) and through the server: each query within 1e-6 of the oracle push
    and of the same query alone."""
    g, og = tiny["g"], tiny["og"]
    G = ahpp.Graph.from_arrays(g, algo=ahpp.AHPP_APP_S, attr_bf16=0)
    try:
        qs = [int(x) for x in synth.draw_queries(g.n_u, 35, seed=78)]
        eps = np.where(np.arange(35) % 2 == 0, 1e-6, 1e-4)
        dense, stats, rc = G.query_batch_dense(qs, eps)
        assert rc == 0
        for i in [0, 1, 17, 33, 34]:
            ref = og.push("apps", ALPHA, BETA, qs[i], float(eps[i]))
            assert np.abs(dense[i].astype(np.float64) - ref.pi).max() <= TOL
            assert abs(stats[i]["rounds"] - ref.stats["rounds"]) <= 1
            assert abs(stats[i]["switch_round"] - ref.stats["switch_round"]) <= 1
            one, st1, _ = G.query_dense(qs[i], float(eps[i]))
            assert np.abs(one - dense[i]).max() <= TOL
        srv = ahpp.Server(G, max_slots=32, rounds_per_step=3, single_max=-1)
        try:
            t = [srv.submit(qs[i], float(eps[i]), 40) for i in range(35)]
            res = [srv.wait(x, 40) for x in t]
        finally:
            srv.stop()
        for i in [0, 17, 34]:
            assert res[i].rc == 0
            check_topk(res[i].nodes, res[i].scores, dense[i], 40, float(eps[i]))
    finally:
        G.close()


def test_empty_batch_and_k_clamped(ahpp, tiny):
    G, g = tiny["G"], tiny["g"]
    assert G.query_batch([], 1e-6, 10) == []
    res = G.query_batch([3, 5], 1e-4, ahpp.AHPP_MAX_K)
    for r in res:
        assert r.nodes.shape[0] == g.n_u
        assert sorted(r.nodes.tolist()) == list(range(g.n_u))
        assert np.all(np.diff(r.scores) <= 0)
    with pytest.raises(ahpp.AhppError) as e:
        G.query_batch([3], 1e-6, ahpp.AHPP_MAX_K + 1)
    assert e.value.code == ahpp.AHPP_EINVAL


def test_device_wait_gives_up_and_context_survives(ahpp, tiny):
    """Failure detection without a fault: a grid barrier that can never fill
    gives up within its bounded spin, reports it, and the context keeps
    working (a query runs afterwards)."""
    gave_up, ctx_ok = ahpp.selftest_wait_timeout(0)
    assert gave_up == 2 and ctx_ok
    r = tiny["G"].query(3, 1e-4, 5)
    assert r.rc == 0 and r.nodes.shape[0] == 5


def test_wait_timeout_at_the_first_barrier_of_each_query_kernel(ahpp, tiny):
    """The same bounded wait inside the query kernels: with the self-test trap
    armed, the launch's first grid barrier (before any round) can never fill,
    every block gives up after its bounded spin, and the call reports
    AHPP_ETIMEOUT instead of a previous call's status; the next call works."""
    torch = pytest.importorskip("torch")
    G, og, lam = tiny["G"], tiny["og"], tiny["lam"]
    q = 3
    ref = og.push("asrp", ALPHA, BETA, q, 1e-6, lam=lam)
    good, _, _ = G.query_dense(q, 1e-6)          # leaves status "converged" behind
    # single query (plain path)
    G.arm_wait_timeout()
    with pytest.raises(ahpp.AhppError) as e:
        G.query_dense(q, 1e-6)
    assert e.value.code == ahpp.AHPP_ETIMEOUT
    # single query into device buffers: the status arrives in the stats
    dev = torch.device("cuda", 0)
    nodes_t = torch.zeros(5, dtype=torch.int32, device=dev)
    scores_t = torch.zeros(5, dtype=torch.float32, device=dev)
    n_t = torch.zeros(1, dtype=torch.int32, device=dev)
    st_t = torch.zeros((1, ahpp.STATS_BYTES), dtype=torch.uint8, device=dev)
    G.arm_wait_timeout()
    G.query_device(q, 1e-6, 5, nodes_t, scores_t, n_t, st_t, None)
    torch.cuda.synchronize()
    assert stats_of(ahpp, st_t)[0]["status"] == 2
    # batched launch (two tiles, ragged): every query reports the wait
    qs = [int(x) for x in synth.draw_queries(tiny["g"].n_u, 40, seed=97)]
    G.arm_wait_timeout()
    out = np.zeros((40, tiny["g"].n_u), np.float32)
    st = (ahpp.Stats * 40)()
    rc = ahpp.lib().ahpp_query_batch_dense(
        G.handle, 40, np.ascontiguousarray(qs, np.uint32).ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
        np.full(40, 1e-6).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), st)
    assert rc == ahpp.AHPP_ETIMEOUT
    assert all(st[i].status == 2 for i in range(40))
    # Algorithm 1 mode
    G.arm_wait_timeout()
    with pytest.raises(ahpp.AhppError) as e:
        G.power_iteration(q, 10)
    assert e.value.code == ahpp.AHPP_ETIMEOUT
    # the trap is one-shot and the graph keeps working
    again, st2, rc = G.query_dense(q, 1e-6)
    assert rc == 0 and st2["status"] == 0
    assert np.abs(again.astype(np.float64) - ref.pi).max() <= TOL
    assert np.abs(again - good).max() <= TOL
    dense, stats, rc = G.query_batch_dense(qs, 1e-6)
    assert rc == 0 and all(s["status"] == 0 for s in stats)


def test_wait_timeout_fails_the_server(ahpp, tiny):
    """A serving step whose wait gives up fails its requests with
    AHPP_ETIMEOUT and stops the server; a new server on the graph works."""
    G = tiny["G"]
    qs = [int(x) for x in synth.draw_queries(tiny["g"].n_u, 40, seed=98)]
    srv = ahpp.Server(G, max_slots=32, rounds_per_step=4, single_max=-1)
    try:
        G.arm_wait_timeout()
        t = srv.submit(qs[0], 1e-6, 5)
        # no timeout on the wait itself (-1): AHPP_ETIMEOUT here is the device's
        rc = ahpp.lib().ahpp_wait(srv._h, t, -1, None, None, None, None)
        assert rc == ahpp.AHPP_ETIMEOUT
        assert "serving loop failed" in ahpp.lib().ahpp_last_error().decode()
    finally:
        srv.stop()
    srv = ahpp.Server(G, max_slots=32, rounds_per_step=4, single_max=-1)
    try:
        t = srv.submit(qs[0], 1e-6, 5)
        r = srv.wait(t, 5)
        assert r.rc == 0 and r.nodes.shape[0] == 5
    finally:
        srv.stop()


def test_graph_cache_round_trip(ahpp, tiny, tmp_path):
    """A saved graph loads back without the build: same sizes and lambda,
    same results; mismatched alpha and truncated, damaged or extended files
    are refused."""
    G, g = tiny["G"], tiny["g"]
    path = str(tmp_path / "tiny.ahppg")
    G.save(path)
    H = ahpp.Graph.load_file(path, attr_bf16=0, lam=tiny["lam"])
    try:
        for key in ("n_u", "n_v", "n_a", "n_e", "n_ea", "graph_bytes", "lambda"):
            assert H.info[key] == G.info[key], key
        qs = [int(x) for x in synth.draw_queries(g.n_u, 40, seed=95)]
        a, sa, _ = G.query_batch_dense(qs, 1e-6)
        b, sb, rc = H.query_batch_dense(qs, 1e-6)
        assert rc == 0 and np.abs(a - b).max() <= 1e-7
        assert [s["rounds"] for s in sa] == [s["rounds"] for s in sb]
        one = H.query(qs[0], 1e-6, 20)
        check = G.query(qs[0], 1e-6, 20)
        assert len(set(one.nodes.tolist()) & set(check.nodes.tolist())) >= 19
    finally:
        H.close()
    with pytest.raises(ahpp.AhppError) as e:
        ahpp.Graph.load_file(path, attr_bf16=0, lam=tiny["lam"], alpha=0.2)
    assert e.value.code == ahpp.AHPP_EINVAL
    data = open(path, "rb").read()
    bad = str(tmp_path / "cut.ahppg")
    open(bad, "wb").write(data[: len(data) // 2])
    with pytest.raises(ahpp.AhppError) as e:
        ahpp.Graph.load_file(bad, attr_bf16=0, lam=tiny["lam"])
    assert e.value.code == ahpp.AHPP_EINVAL
    with pytest.raises(ahpp.AhppError):
        ahpp.Graph.load_file(str(tmp_path / "missing.ahppg"), attr_bf16=0, lam=tiny["lam"])
    # one flipped byte in the arrays, or bytes after the checksum: refused
    flipped = bytearray(data)
    flipped[len(data) * 3 // 4] ^= 0x10
    for name, blob in (("flip.ahppg", bytes(flipped)), ("tail.ahppg", data + b"\0" * 8)):
        bad = str(tmp_path / name)
        open(bad, "wb").write(blob)
        with pytest.raises(ahpp.AhppError) as e:
            ahpp.Graph.load_file(bad, attr_bf16=0, lam=tiny["lam"])
        assert e.value.code == ahpp.AHPP_EINVAL
    # the intact file still loads after the refusals
    ahpp.Graph.load_file(path, attr_bf16=0, lam=tiny["lam"]).close()


def test_graph_cache_keeps_the_lambda_estimate(ahpp, tmp_path):
    """A graph loaded with the Theorem 3 estimate keeps it through the cache
    (no new lambda run) when loaded with the same lambda_T."""
    g = synth.make_graph(**synth.TINY)
    G = ahpp.Graph.from_arrays(g, attr_bf16=0)
    path = str(tmp_path / "lam.ahppg")
    try:
        G.save(path)
        H = ahpp.Graph.load_file(path, attr_bf16=0)
        try:
            assert H.info["lambda"] == G.info["lambda"] and H.info["lambda_T"] == G.info["lambda_T"]
        finally:
            H.close()
    finally:
        G.close()
