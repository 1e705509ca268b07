"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value the
paper prints (the worked example of Section 2.1), transition rows derived by
hand (tests/golden/hand_graph.txt), closed forms, a different algorithm for
the same quantity (series of Eq. 3 vs. linear solve vs. Power Iteration vs.
the sampled walk of Lemma 1), or a theorem's invariant (Lemma 3,
Theorems 2 and 3, mass conservation).
"""
import math

import numpy as np
import pytest

import oracle
from golden_io import load
from paper_2512_11606_gb300 import synth

ALPHA, BETA = 0.15, 0.35


def graph_of(fx):
    return synth.GraphArrays(fx.n_u, fx.n_v, fx.n_a, fx.e_u, fx.e_v,
                             np.asarray(fx.e_w, np.float32), fx.ea_u, fx.ea_a,
                             np.asarray(fx.ea_w, np.float32))


def frac_row(row):
    return np.array([float(x) for x in row])


@pytest.fixture(scope="module")
def tiny():
    g = synth.make_graph(**synth.TINY)
    og = oracle.OracleGraph.from_arrays(g)
    _, _, P = oracle.dense_matrices_of(g, BETA)
    Pi = oracle.pi_matrix(P, ALPHA)
    lam, _ = og.lambda_estimate(ALPHA, BETA)
    q = int(synth.draw_queries(g.n_u, 1)[0])
    return dict(g=g, og=og, P=P, Pi=Pi, lam=lam, q=q)


# ----------------------------------------------------------- worked example

def test_worked_example_dense_row():
    """Example 1 (Section 2.1): P_S[u1,u2] = 3/8, P_S[u1,u3] = 1/8 (+ implied)."""
    fx = load("worked_example.txt")
    P_S, _, _ = oracle.dense_matrices_of(graph_of(fx), 0.0)
    np.testing.assert_allclose(P_S[0], frac_row(fx.ps_rows[0]), rtol=0, atol=1e-15)


@pytest.mark.parametrize("algo", ["app", "asrp"])
def test_worked_example_one_push_round(algo):
    """One round of Algorithm 3/4 from u1 with beta = 0 leaves r = (1-a) P_S[u1, .]."""
    fx = load("worked_example.txt")
    og = oracle.OracleGraph.from_arrays(graph_of(fx))
    res = og.push(algo, ALPHA, 0.0, 0, 1e-9, lam=1.0, max_rounds=1)
    assert res.stats["rounds"] == 1 and res.rc == 1
    np.testing.assert_allclose(res.r_u, (1 - ALPHA) * frac_row(fx.ps_rows[0]), atol=1e-15)
    assert res.pi[0] == pytest.approx(ALPHA, abs=1e-15)
    assert np.all(res.pi[1:] == 0)


# -------------------------------------------------------- hand-derived rows

def test_hand_graph_dense_rows():
    fx = load("hand_graph.txt")
    P_S, P_A, _ = oracle.dense_matrices_of(graph_of(fx), BETA)
    for i, row in fx.ps_rows.items():
        np.testing.assert_allclose(P_S[i], frac_row(row), atol=1e-15)
    for i, row in fx.pa_rows.items():
        np.testing.assert_allclose(P_A[i], frac_row(row), atol=1e-15)


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("beta", [0.0, 0.25, 0.35, 1.0])
def test_hand_graph_one_push_round(q, beta):
    """The C oracle's two-hop push reproduces the hand rows of (1-b)P_S + b P_A."""
    fx = load("hand_graph.txt")
    og = oracle.OracleGraph.from_arrays(graph_of(fx))
    res = og.push("asrp", ALPHA, beta, q, 1e-9, lam=1.0, max_rounds=1)
    row = (1 - beta) * frac_row(fx.ps_rows[q]) + beta * frac_row(fx.pa_rows[q])
    np.testing.assert_allclose(res.r_u, (1 - ALPHA) * row, atol=1e-15)


def test_pins_catch_planted_mistakes():
    """Plausible mistakes in the dense builder fail the hand pins."""
    fx = load("hand_graph.txt")
    g = graph_of(fx)
    WA = np.zeros((g.n_u, g.n_a))
    np.add.at(WA, (g.ea_u.astype(int), g.ea_a.astype(int)), g.ea_w.astype(float))
    good = frac_row(fx.pa_rows[0])
    # normalisers swapped (column sum on the left hop, row sum on the right)
    swapped = (WA / WA.sum(0)[None, :]) @ (WA / WA.sum(1)[:, None]).T
    # transposed operand (column of P_A instead of its row)
    _, P_A, _ = oracle.dense_matrices_of(g, BETA)
    assert not np.allclose(swapped[0], good)
    assert not np.allclose(P_A[:, 0], good)
    # a dropped attribute term (beta part lost) changes the pushed round
    og = oracle.OracleGraph.from_arrays(g)
    res = og.push("asrp", ALPHA, 0.35, 0, 1e-9, lam=1.0, max_rounds=1)
    only_s = (1 - ALPHA) * (0.65 * frac_row(fx.ps_rows[0]))
    assert not np.allclose(res.r_u, only_s)


# --------------------------------------------------------------- closed forms

def hub_graph(n):
    """One V node joined to every U node, one attribute shared by all: P = J/n."""
    u = np.arange(n, dtype=np.uint32)
    z = np.zeros(n, dtype=np.uint32)
    one = np.ones(n, dtype=np.float32)
    return synth.GraphArrays(n, 1, 1, u, z, one, u, z, one)


@pytest.mark.parametrize("n", [2, 5, 17])
def test_closed_form_uniform_chain(n):
    """P = J/n gives pi(u,u) = a + (1-a)/n and pi(u,j) = (1-a)/n (j != u)."""
    g = hub_graph(n)
    og = oracle.OracleGraph.from_arrays(g)
    want = np.full(n, (1 - ALPHA) / n)
    want[1] += ALPHA
    _, _, P = oracle.dense_matrices_of(g, BETA)
    np.testing.assert_allclose(P, np.full((n, n), 1.0 / n), atol=1e-15)
    np.testing.assert_allclose(oracle.exact_dense(P, ALPHA, 1), want, atol=1e-14)
    np.testing.assert_allclose(og.power_iteration(ALPHA, BETA, 1, 400), want, atol=1e-14)
    eps = 1e-10
    for algo in ("app", "asrp"):
        res = og.push(algo, ALPHA, BETA, 1, eps, lam=1.0)
        assert res.rc == 0
        assert np.all(want - res.pi >= -1e-15) and np.all(want - res.pi <= eps * 1.0001)


def hub_trajectory(n, eps, lam, rule):
    """ASRP on the hub graph, worked out by hand.

    Every round after the first pushes all n U nodes with equal residues, so
    after round k each residue is (1-a)^k / n.  Round 1 pushes q alone: its
    two entries plus the V and A flushes (n each) give n_p = 2n + 2; every
    later round adds 2n pushed entries and 2n flushed ones, so
    n_p(k) = 4nk - 2n + 2.  The loop ends after the first round R with
    (1-a)^R / n <= eps_f (eps_f = eps / lam): R = ceil(L) with
    L = log_{1/(1-a)} (1 / (n eps_f)).  The switch test after asynchronous
    round k compares n_p(k) with the budget 2(|E| + |E_A|) = 4n times
      rule 0 (the budget of Theorem 1's proof): max(0, L - k), which n_p(k)
              reaches from k >= L/2 + 1/4 - 1/(4n) on;
      rule 1 (the formula as printed): log_{1/(1-a)} (n / lam) + k, which
              n_p(k) reaches at every k or at none: iff that log is at most
              (1 - n) / (2n).
    Returns (rounds, switch_round, the thresholds that decide them)."""
    lg = math.log(1 / (1 - ALPHA))
    L = math.log(lam / (n * eps)) / lg
    R = math.ceil(L)
    if rule == 0:
        ks = max(1, math.ceil(L / 2 + 0.25 - 0.25 / n))
        cuts = [L, L / 2 + 0.25 - 0.25 / n]
    else:
        L1 = math.log(n / lam) / lg
        ks = 1 if L1 <= (1 - n) / (2 * n) else None
        cuts = [L, L1 - (1 - n) / (2 * n)]
    sr = ks + 1 if ks is not None and ks <= R else 0
    return R, sr, cuts


@pytest.mark.parametrize("n,eps,lam,rule", [(5, 1e-6, 3.0, 0), (17, 1e-9, 50.0, 0), (2, 1e-4, 1.5, 0),
                                            (5, 1e-6, 100.0, 1), (5, 1e-6, 3.0, 1)])
def test_asrp_trajectory_closed_form_on_hub_graph(n, eps, lam, rule):
    """The ASRP switch and termination, n_p accounting, traces and the final
    reserves on P = J/n against the trajectory derived by hand."""
    R, sr, cuts = hub_trajectory(n, eps, lam, rule)
    for c in cuts:              # no decision sits on a rounding boundary
        assert abs(c - round(c)) > 1e-6 or abs(c) > 1e6
    og = oracle.OracleGraph.from_arrays(hub_graph(n))
    q = n // 2
    res = og.push("asrp", ALPHA, BETA, q, eps, lam=lam, switch_rule=rule)
    check_hub_run(res, n, q, R, sr)


@pytest.mark.parametrize("n,eps", [(5, 1e-6), (17, 1e-9), (2, 3e-4)])
def test_app_trajectory_closed_form_on_hub_graph(n, eps):
    """APP on P = J/n: every U node has |N(u)| + |A(u)| = 2 and
    r_max = eps / (|E| + |E_A|) = eps / (2n), so the threshold is eps / n and
    the run ends after the first round R with (1-a)^R <= eps; the rounds
    push as in ASRP's (n_p, traces, reserves) without a phase switch."""
    L = math.log(1 / eps) / math.log(1 / (1 - ALPHA))
    assert abs(L - round(L)) > 1e-6
    R = math.ceil(L)
    og = oracle.OracleGraph.from_arrays(hub_graph(n))
    q = n - 1
    res = og.push("app", ALPHA, BETA, q, eps)
    check_hub_run(res, n, q, R, 0)


@pytest.mark.parametrize("n,eps", [(5, 1e-6), (17, 1e-9), (2, 3e-4)])
def test_apps_trajectory_closed_form_on_hub_graph(n, eps):
    """APP(S) (APP with ASRP's synchronous switch, the ablation arm of Exp-2)
    on P = J/n: every node has |N(u)| + |A(u)| = 2, so APP's threshold is
    r_max * 2 = eps / n for all of them and the largest residue in units of
    its threshold is M / 2 / r_max = M n / eps.  The run is therefore ASRP's
    hand trajectory with eps_f = eps / n (lambda = n) under the read budget:
    the same switch round, rounds, n_p, traces and reserves."""
    R, sr, cuts = hub_trajectory(n, eps, float(n), 0)
    for c in cuts:
        assert abs(c - round(c)) > 1e-6 or abs(c) > 1e6
    og = oracle.OracleGraph.from_arrays(hub_graph(n))
    q = n // 3
    res = og.push("apps", ALPHA, BETA, q, eps)
    check_hub_run(res, n, q, R, sr)
    assert sr > 0 or R <= 2


def check_hub_run(res, n, q, R, sr):
    s, t = res.stats, res.trace
    assert res.rc == 0
    assert s["rounds"] == R and s["switch_round"] == sr
    k = np.arange(1, R + 1)
    assert t["frontier"].tolist() == [1] + [n] * (R - 1)
    assert t["n_p"].tolist() == (4 * n * k - 2 * n + 2).tolist()
    assert s["n_p"] == 4 * n * R - 2 * n + 2 and s["pushes"] == 1 + n * (R - 1)
    np.testing.assert_allclose(t["max_r"], (1 - ALPHA) ** k / n, rtol=1e-12)
    want_phase = [0] * R if sr == 0 else [0] * (sr - 1) + [1] * (R - sr + 1)
    assert t["phase"].tolist() == want_phase[:R]
    share = ALPHA * sum((1 - ALPHA) ** j for j in range(1, R)) / n
    want = np.full(n, share)
    want[q] += ALPHA
    np.testing.assert_allclose(res.pi, want, rtol=1e-12)
    np.testing.assert_allclose(res.r_u, np.full(n, (1 - ALPHA) ** R / n), rtol=1e-12)


def small_random_graph(seed, n_u=8, n_v=6, n_e=18, n_a=4, m=2):
    rng = np.random.default_rng(seed)
    pairs = set()
    # every node gets at least one edge
    for u in range(n_u):
        pairs.add((u, int(rng.integers(n_v))))
    for v in range(n_v):
        pairs.add((int(rng.integers(n_u)), v))
    while len(pairs) < n_e:
        pairs.add((int(rng.integers(n_u)), int(rng.integers(n_v))))
    e = np.array(sorted(pairs))
    ew = rng.uniform(0.5, 2.0, size=e.shape[0]).astype(np.float32)
    au = np.repeat(np.arange(n_u), m)
    aa = np.concatenate([rng.choice(n_a, size=m, replace=False) for _ in range(n_u)])
    aw = rng.uniform(0.1, 1.0, size=au.shape[0]).astype(np.float32)
    return synth.GraphArrays(n_u, n_v, n_a, e[:, 0].astype(np.uint32),
                             e[:, 1].astype(np.uint32), ew, au.astype(np.uint32),
                             aa.astype(np.uint32), aw)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_series_solve_and_power_iteration_agree(seed):
    """Eq. 3 summed term by term = the linear solve = Algorithm 1."""
    g = small_random_graph(seed)
    _, _, P = oracle.dense_matrices_of(g, BETA)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-14)
    og = oracle.OracleGraph.from_arrays(g)
    for q in range(g.n_u):
        ex = oracle.exact_dense(P, ALPHA, q)
        np.testing.assert_allclose(oracle.series_sum(P, ALPHA, q, 400), ex, atol=1e-13)
        np.testing.assert_allclose(og.power_iteration(ALPHA, BETA, q, 250), ex, atol=1e-13)
        assert ex.sum() == pytest.approx(1.0, abs=1e-13)


def test_monte_carlo_walks_match_exact():
    """Lemma 1: the stop distribution of the sampled walk is pi(q, .)."""
    g = small_random_graph(5)
    _, _, P = oracle.dense_matrices_of(g, BETA)
    q, n = 3, 2_000_000
    emp = oracle.monte_carlo_walks(g, ALPHA, BETA, q, n)
    ex = oracle.exact_dense(P, ALPHA, q)
    sigma = np.sqrt(ex * (1 - ex) / n)
    assert np.all(np.abs(emp - ex) <= 5 * sigma + 1e-6), (emp, ex)


def test_beta_selects_terms():
    """beta = 0 ignores attribute weights; beta = 1 ignores edge weights."""
    g = small_random_graph(3)
    g2 = synth.GraphArrays(g.n_u, g.n_v, g.n_a, g.e_u, g.e_v, g.e_w, g.ea_u, g.ea_a,
                           (g.ea_w * np.linspace(0.3, 3.0, g.ea_w.shape[0])).astype(np.float32))
    g3 = synth.GraphArrays(g.n_u, g.n_v, g.n_a, g.e_u, g.e_v,
                           (g.e_w * np.linspace(0.3, 3.0, g.e_w.shape[0])).astype(np.float32),
                           g.ea_u, g.ea_a, g.ea_w)
    a, b, c = (oracle.OracleGraph.from_arrays(x) for x in (g, g2, g3))
    np.testing.assert_allclose(a.power_iteration(ALPHA, 0.0, 2, 200),
                               b.power_iteration(ALPHA, 0.0, 2, 200), atol=1e-15)
    np.testing.assert_allclose(a.power_iteration(ALPHA, 1.0, 2, 200),
                               c.power_iteration(ALPHA, 1.0, 2, 200), atol=1e-15)
    assert not np.allclose(a.power_iteration(ALPHA, BETA, 2, 200),
                           b.power_iteration(ALPHA, BETA, 2, 200))


def test_disconnected_components_have_zero_cross_scores():
    g1 = small_random_graph(7, n_u=5, n_v=4, n_e=9, n_a=3, m=1)
    g2 = small_random_graph(8, n_u=4, n_v=3, n_e=7, n_a=2, m=1)
    g = synth.GraphArrays(
        9, 7, 5,
        np.concatenate([g1.e_u, g2.e_u + 5]).astype(np.uint32),
        np.concatenate([g1.e_v, g2.e_v + 4]).astype(np.uint32),
        np.concatenate([g1.e_w, g2.e_w]),
        np.concatenate([g1.ea_u, g2.ea_u + 5]).astype(np.uint32),
        np.concatenate([g1.ea_a, g2.ea_a + 3]).astype(np.uint32),
        np.concatenate([g1.ea_w, g2.ea_w]))
    og = oracle.OracleGraph.from_arrays(g)
    _, _, P = oracle.dense_matrices_of(g, BETA)
    ex = oracle.exact_dense(P, ALPHA, 1)
    assert np.all(ex[5:] == 0)
    res = og.push("asrp", ALPHA, BETA, 1, 1e-9, lam=1.0)
    assert np.all(res.pi[5:] == 0) and np.all(res.r_u[5:] == 0)


def test_duplicate_pairs_are_merged():
    g = small_random_graph(4)
    dup = synth.GraphArrays(g.n_u, g.n_v, g.n_a,
                            np.concatenate([g.e_u, g.e_u[:3]]),
                            np.concatenate([g.e_v, g.e_v[:3]]),
                            np.concatenate([g.e_w, g.e_w[:3]]),
                            g.ea_u, g.ea_a, g.ea_w)
    merged_w = g.e_w.copy()
    merged_w[:3] *= 2
    single = synth.GraphArrays(g.n_u, g.n_v, g.n_a, g.e_u, g.e_v, merged_w,
                               g.ea_u, g.ea_a, g.ea_w)
    a, b = oracle.OracleGraph.from_arrays(dup), oracle.OracleGraph.from_arrays(single)
    assert a.n_e == g.n_e
    np.testing.assert_allclose(a.power_iteration(ALPHA, BETA, 0, 100),
                               b.power_iteration(ALPHA, BETA, 0, 100), atol=1e-15)


def test_invalid_inputs_raise():
    g = small_random_graph(1)
    bad = synth.GraphArrays(g.n_u, g.n_v, g.n_a, g.e_u, g.e_v, -g.e_w, g.ea_u, g.ea_a, g.ea_w)
    with pytest.raises(ValueError):
        oracle.OracleGraph.from_arrays(bad)
    og = oracle.OracleGraph.from_arrays(g)
    with pytest.raises(ValueError):
        og.push("asrp", ALPHA, BETA, g.n_u, 1e-6, lam=1.0)
    with pytest.raises(ValueError):
        og.push("asrp", ALPHA, BETA, 0, 0.0, lam=1.0)


def test_dangling_rows_leak_and_conserve():
    """A U node without attributes drops the beta share (reading of Eq. 2)."""
    g = small_random_graph(9)
    keep = g.ea_u != 2
    g2 = synth.GraphArrays(g.n_u, g.n_v, g.n_a, g.e_u, g.e_v, g.e_w,
                           g.ea_u[keep], g.ea_a[keep], g.ea_w[keep])
    og = oracle.OracleGraph.from_arrays(g2)
    res = og.push("asrp", ALPHA, BETA, 2, 1e-10, lam=1.0)
    s = res.stats
    assert s["leak"] > 0
    assert s["reserve_sum"] + s["resid_sum"] + s["leak"] == pytest.approx(1.0, abs=1e-12)
    _, _, P = oracle.dense_matrices_of(g2, BETA)
    assert P[2].sum() == pytest.approx(1 - BETA, abs=1e-15)
    ex = oracle.exact_dense(P, ALPHA, 2)
    assert np.all(ex - res.pi >= -1e-15) and np.all(ex - res.pi <= 1e-10)


# ------------------------------------------------ theorems on the tiny graph

def test_tiny_no_dangling_and_row_stochastic(tiny):
    np.testing.assert_allclose(tiny["P"].sum(axis=1), 1.0, atol=1e-12)


def test_lambda_bounds_column_sums(tiny):
    """Theorem 3: lambda >= max_i sum_j pi(u_j, u_i)."""
    colsum = tiny["Pi"].sum(axis=0).max()
    assert tiny["lam"] >= colsum
    # the bound is tight up to the tail term |U| (1-alpha)^T <= 0.01
    assert tiny["lam"] <= colsum + 0.0101


@pytest.mark.parametrize("n", [3, 11])
def test_lambda_estimate_closed_form_on_weighted_hub(n):
    """Theorem 3's estimate on a weighted hub: U node i joined to the one V
    node with weight w_i and to the one attribute with weight x_i.  Then every
    row of P is mu = (1-b) w/W + b x/X (Eq. 1 and Eq. 2 with one middle node),
    so 1 P^l = n mu for l >= 1 and
        pi_T = a + n mu ((1-a) - (1-a)^T),
        lambda = max pi_T + n (1-a)^T,
    with T = ceil(ln(100 n) / ln(1/(1-a))); the exact column sums of Pi are
    a + (1-a) n mu, below lambda."""
    rng = np.random.default_rng(n)
    w = rng.uniform(0.5, 2.0, n).astype(np.float32)
    x = rng.uniform(0.1, 1.0, n).astype(np.float32)
    u = np.arange(n, dtype=np.uint32)
    z = np.zeros(n, dtype=np.uint32)
    g = synth.GraphArrays(n, 1, 1, u, z, w, u, z, x)
    og = oracle.OracleGraph.from_arrays(g)
    wd, xd = w.astype(np.float64), x.astype(np.float64)
    mu = (1 - BETA) * wd / wd.sum() + BETA * xd / xd.sum()
    T = math.ceil(math.log(100 * n) / math.log(1 / (1 - ALPHA)))
    tail = (1 - ALPHA) ** T
    want_piT = ALPHA + n * mu * ((1 - ALPHA) - tail)
    lam, piT = og.lambda_estimate(ALPHA, BETA)
    np.testing.assert_allclose(piT, want_piT, rtol=1e-12)
    assert lam == pytest.approx(want_piT.max() + n * tail, rel=1e-12)
    _, _, P = oracle.dense_matrices_of(g, BETA)
    np.testing.assert_allclose(P, np.tile(mu, (n, 1)), rtol=1e-12)
    colsum = oracle.pi_matrix(P, ALPHA).sum(axis=0)
    np.testing.assert_allclose(colsum, ALPHA + (1 - ALPHA) * n * mu, rtol=1e-10)
    assert lam >= colsum.max()


def test_lemma3_invariant_every_round(tiny):
    """Lemma 3: pi(q, .) = pi_hat + r Pi after every round (APP and ASRP)."""
    og, Pi, q, lam = tiny["og"], tiny["Pi"], tiny["q"], tiny["lam"]
    exact = Pi[q]
    for algo in ("asrp", "app"):
        full = og.push(algo, ALPHA, BETA, q, 1e-6, lam=lam)
        R = full.stats["rounds"]
        for k in sorted({1, 2, 3, 5, R // 2, R}):
            res = og.push(algo, ALPHA, BETA, q, 1e-6, lam=lam, max_rounds=k)
            np.testing.assert_allclose(res.pi + res.r_u @ Pi, exact, atol=1e-12)
            assert np.all(res.pi >= 0) and np.all(res.r_u >= 0)


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_theorem2_error_bound(tiny, eps):
    """Theorem 2: 0 <= pi - pi_hat <= eps with the certified lambda; APP too."""
    og, Pi, q, lam = tiny["og"], tiny["Pi"], tiny["q"], tiny["lam"]
    exact = Pi[q]
    for algo in ("asrp", "app", "apps"):
        res = og.push(algo, ALPHA, BETA, q, eps, lam=lam)
        assert res.rc == 0
        err = exact - res.pi
        assert err.min() >= -1e-14 and err.max() <= eps, (algo, err.min(), err.max())
    fp = og.forward_push(ALPHA, BETA, q, eps)
    err = exact - fp.pi
    assert err.min() >= -1e-14 and err.max() <= eps


def test_mass_conservation_per_round(tiny):
    og, q, lam = tiny["og"], tiny["q"], tiny["lam"]
    res = og.push("asrp", ALPHA, BETA, q, 1e-6, lam=lam)
    t = res.trace
    np.testing.assert_allclose(t["sum_pi"] + t["sum_r"], 1.0, atol=1e-12)
    assert np.all(np.diff(t["sum_pi"]) >= 0)
    assert np.all(np.diff(t["n_p"].astype(np.int64)) > 0)


def test_asrp_switch_and_termination_consistency(tiny):
    """Rounds after the switch are synchronous; the loop ends at max r <= eps_f."""
    og, q, lam = tiny["og"], tiny["q"], tiny["lam"]
    eps = 1e-6
    res = og.push("asrp", ALPHA, BETA, q, eps, lam=lam)
    s, t = res.stats, res.trace
    assert s["max_resid"] <= eps / lam
    assert np.all(t["max_r"][:-1] > eps / lam)
    if s["switch_round"]:
        sr = s["switch_round"]
        assert np.all(t["phase"][: sr - 1] == 0) and np.all(t["phase"][sr - 1:] == 1)
        # the budget test that fired: n_p >= 2(|E|+|E_A|) log_{1/(1-a)}(M/eps_f)
        EE = og.n_e + og.n_ea
        M = t["max_r"][sr - 2]
        budget = 2 * EE * max(0.0, math.log(M / (eps / lam)) / math.log(1 / (1 - ALPHA)))
        assert t["n_p"][sr - 2] >= budget
    never = og.push("asrp", ALPHA, BETA, q, eps, lam=lam, switch_rule=2)
    assert never.stats["switch_round"] == 0
    np.testing.assert_allclose(never.pi, res.pi, atol=eps)


def test_asrp_selection_rule_of_each_phase(tiny):
    """Algorithm 4 pushes, in an asynchronous round, exactly the U nodes whose
    residue exceeds eps_f and, in a synchronous round, every U node with a
    positive residue.  The residues before round j come from a second run
    stopped after j - 1 rounds."""
    og, q, lam = tiny["og"], tiny["q"], tiny["lam"]
    eps = 1e-6
    eps_f = eps / lam
    full = og.push("asrp", ALPHA, BETA, q, eps, lam=lam)
    sr, R = full.stats["switch_round"], full.stats["rounds"]
    assert 2 < sr < R
    checked = {0: 0, 1: 0}
    for j in sorted({2, 3, sr - 1, sr, sr + 1, R}):
        before = og.push("asrp", ALPHA, BETA, q, eps, lam=lam, max_rounds=j - 1)
        assert before.rc == 1 and before.stats["rounds"] == j - 1
        sync = j >= sr
        want = int((before.r_u > 0).sum()) if sync else int((before.r_u > eps_f).sum())
        assert full.trace["frontier"][j - 1] == want, (j, sync)
        checked[int(sync)] += 1
    assert checked[0] and checked[1]
    # near the end the synchronous frontier is wider than the asynchronous
    # rule would give (positive residues at or below eps_f are pushed too)
    wider = False
    for j in range(R, max(sr, R - 6), -1):
        before = og.push("asrp", ALPHA, BETA, q, eps, lam=lam, max_rounds=j - 1)
        n_pos, n_above = int((before.r_u > 0).sum()), int((before.r_u > eps_f).sum())
        assert full.trace["frontier"][j - 1] == n_pos
        if n_pos > n_above:
            wider = True
            break
    assert wider


def test_apps_phases_and_stopping_rule(tiny):
    """APP(S): asynchronous rounds push exactly the nodes above APP's
    per-node threshold r_max (|N(u)| + |A(u)|), synchronous rounds every
    positive residue; the switch fires on the budget in APP's units; the run
    stops on APP's test (no residue above its threshold) and ends earlier
    than APP alone on the tiny graph."""
    og, q = tiny["og"], tiny["q"]
    eps = 1e-6
    EE = og.n_e + og.n_ea
    r_max = eps / EE
    g = tiny["g"]              # distinct pairs only (synth merges duplicates), so counts are tuples
    cnt = (np.bincount(g.e_u, minlength=g.n_u) + np.bincount(g.ea_u, minlength=g.n_u)).astype(np.float64)
    full = og.push("apps", ALPHA, BETA, q, eps)
    s, t = full.stats, full.trace
    sr, R = s["switch_round"], s["rounds"]
    assert 2 < sr < R
    for j in sorted({2, 3, sr - 1, sr, sr + 1, R}):
        before = og.push("apps", ALPHA, BETA, q, eps, max_rounds=j - 1)
        sync = j >= sr
        want = int((before.r_u > 0).sum()) if sync else int((before.r_u > r_max * cnt).sum())
        assert t["frontier"][j - 1] == want, (j, sync)
    # the budget test that fired, with M' = max r(u) / (|N(u)| + |A(u)|)
    before = og.push("apps", ALPHA, BETA, q, eps, max_rounds=sr - 1)
    mrel = (before.r_u[cnt > 0] / cnt[cnt > 0]).max()
    budget = 2 * EE * max(0.0, math.log(mrel / r_max) / math.log(1 / (1 - ALPHA)))
    assert t["n_p"][sr - 2] >= budget
    assert np.all(full.r_u <= r_max * cnt)
    app = og.push("app", ALPHA, BETA, q, eps)
    assert R < app.stats["rounds"]


def test_asrp_topk_precision_against_exact(tiny):
    """The measure of Fig. 7: the top-k of ASRP at eps = 1e-6 against the
    top-k of exact AHPP (a row of the dense Pi), nodes within 2 eps of the
    exact k-th score counted as interchangeable (ties, C-8)."""
    og, Pi, lam = tiny["og"], tiny["Pi"], tiny["lam"]
    eps = 1e-6
    for q in synth.draw_queries(og.n_u, 3, seed=7):
        exact = Pi[int(q)]
        res = og.push("asrp", ALPHA, BETA, int(q), eps, lam=lam)
        for k in (10, 50, 100):
            kth = np.sort(exact)[::-1][k - 1]
            ok = set(np.where(exact >= kth - 2 * eps)[0].tolist())
            got = oracle.topk(res.pi, k)[0].tolist()
            assert len(set(got) & ok) / k >= 0.99, (int(q), k)


def test_topk_matches_sorting(tiny):
    rng = np.random.default_rng(3)
    s = np.round(rng.random(500), 2)            # many ties
    nodes, vals = oracle.topk(s, 50)
    order = np.lexsort((np.arange(500), -s))[:50]
    assert np.array_equal(nodes, order) and np.array_equal(vals, s[order])


def test_forward_push_fifo_hand_trace():
    """Algorithm 2's FIFO order, traced by hand (tests/golden/forward_push_fifo.txt):
    the reserves, residues and push count after the queue empties.  A stack
    order, or a node re-queued before its neighbours, ends elsewhere."""
    fx = load("forward_push_fifo.txt")
    og = oracle.OracleGraph(fx.n_u, fx.n_v, fx.n_a, fx.e_u, fx.e_v, fx.e_w, fx.ea_u, fx.ea_a, fx.ea_w)
    alpha, beta, eps, q = (float(x) for x in fx.kv["fp_params"])
    res = og.forward_push(alpha, beta, int(q), eps)
    assert res.rc == 0 and res.stats["pushes"] == int(fx.kv["fp_pushes"][0])
    assert list(res.pi) == [float(x) for x in fx.kv["fp_pi"]]          # dyadic: exact in FP64
    assert list(res.r_u) == [float(x) for x in fx.kv["fp_r"]]


@pytest.mark.parametrize("algo", ["asrp", "app", "apps"])
def test_push_resumed_in_pieces_is_the_same_run(tiny, algo):
    """A push advanced a few rounds at a time from a kept state (the bounded
    steps of the bench's CPU arm) performs exactly the rounds of one
    uninterrupted run: identical reserves, residues and counters."""
    og, q, lam = tiny["og"], tiny["q"], tiny["lam"]
    whole = og.push(algo, ALPHA, BETA, q, 1e-6, lam=lam)
    r = og.push_start(q)
    rc, pieces = 1, 0
    while rc == 1:
        rc = og.push_resume(r, algo, ALPHA, BETA, 1e-6, lam=lam, rounds=3)
        pieces += 1
    assert rc == 0 and pieces > 3
    assert np.array_equal(r.pi, whole.pi) and np.array_equal(r.r_u, whole.r_u)
    for key in ("rounds", "switch_round", "n_p", "pushes", "leak", "reserve_sum", "resid_sum"):
        assert r.stats[key] == whole.stats[key], key
