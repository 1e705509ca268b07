"""Seeded synthetic attributed bipartite graphs and query draws.

This module is the input recipe shared by the CUDA path's tests/bench and by
the CPU oracle's tests.  It holds none of the method's arithmetic: it only
draws a graph G = (U, V, E, A, E_A) (Section 2.1) with power-law degrees on
both sides and a sparse node-attribute matrix, and query nodes.

All randomness comes from numpy's counter-based Philox bit generator
(Philox-4x64-10), keyed by (seed, stream) so every array is reproducible on
any machine and in any order of calls.

Recipe (the stand-ins for the paper's datasets, which are not available):
  * degrees: d ~ Zipf(gamma) (P(d) ∝ d^-gamma, d >= 1), capped at the size of
    the opposite side, rescaled to sum to |E| (floor, then the remainder is
    handed out one stub at a time with probability ∝ degree), d >= 1;
  * pairing: configuration-model stub matching (the V stubs are shuffled);
    duplicate (u, v) pairs are dropped and the edge set is topped up to |E|
    by further degree-proportional draws, so every node keeps degree >= 1;
  * edge weights: unit, or uniform(0.5, 1.5), delivered as float32;
  * attributes: each U node gets m distinct attributes (uniform popularity,
    or Zipf popularity when attr_zipf is given) with uniform(0,1] or
    lognormal(0,1) weights, row-normalised in float64 and delivered as
    float32; with bf16=True the weights are rounded to the nearest
    bfloat16-representable float32 (round-to-nearest-even) so that a
    consumer that stores them as bfloat16 loses nothing.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Stream ids under one seed: each array of a graph draws from its own stream.
_S_DEG_U, _S_DEG_V, _S_PAIR, _S_TOPUP, _S_EW, _S_ATTR, _S_AW, _S_QUERY = range(8)


def rng_for(seed: int, stream: int) -> np.random.Generator:
    """Philox-4x64-10 generator keyed by (seed, stream)."""
    key = np.array([seed & (2**64 - 1), stream & (2**64 - 1)], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


@dataclass
class GraphArrays:
    """COO arrays of an attributed bipartite graph (caller-side input)."""
    n_u: int
    n_v: int
    n_a: int
    e_u: np.ndarray          # uint32 [|E|]
    e_v: np.ndarray          # uint32 [|E|]
    e_w: np.ndarray          # float32 [|E|], > 0
    ea_u: np.ndarray         # uint32 [|E_A|]
    ea_a: np.ndarray         # uint32 [|E_A|]
    ea_w: np.ndarray         # float32 [|E_A|], > 0
    meta: dict = field(default_factory=dict)

    @property
    def n_e(self) -> int:
        return int(self.e_u.shape[0])

    @property
    def n_ea(self) -> int:
        return int(self.ea_u.shape[0])


# Workload shapes (sizes, exponents, weight laws) of the synthetic stand-ins.
TINY = dict(n_u=2000, n_v=3000, n_e=20000, gamma_u=2.1, gamma_v=2.1,
            edge_w="unit", n_a=500, m=10, attr_w="uniform", bf16=False, seed=1)
MEDIUM = dict(n_u=1_000_000, n_v=500_000, n_e=20_000_000, gamma_u=2.1, gamma_v=2.1,
              edge_w="uniform_0.5_1.5", n_a=10_000, m=20, attr_w="lognormal",
              bf16=False, seed=2)
MEDIUM_BF16 = dict(MEDIUM, bf16=True)
LARGE = dict(n_u=5_000_000, n_v=5_000_000, n_e=200_000_000, gamma_u=2.0, gamma_v=2.0,
             edge_w="uniform_0.5_1.5", n_a=50_000, m=30, attr_w="lognormal",
             bf16=True, seed=3)


def _choice_counts(rng: np.random.Generator, p: np.ndarray, size: int) -> np.ndarray:
    """How often each index is drawn by size draws with probabilities p.

    The same draws as Generator.choice(len(p), size, p=p) (one uniform per
    draw, located in the normalised cumulative sum), counted per index; the
    uniforms are located in sorted order, which leaves the counts unchanged
    and keeps the lookups cache-friendly."""
    cdf = p.cumsum()
    cdf /= cdf[-1]
    u = np.sort(rng.random(size))
    return np.bincount(_searchsorted(cdf, u, right=True), minlength=p.shape[0])


# The large graph's arrays hold 10^8 elements; torch's CPU sort and binary
# search run on all host cores where numpy's run on one.  Both are exact: a
# stable sort is unique, and a binary search has one answer.
def _stable_argsort(a: np.ndarray) -> np.ndarray:
    """The stable sorting permutation of a (equal values keep their order)."""
    import torch
    return torch.sort(torch.from_numpy(np.ascontiguousarray(a)), stable=True).indices.numpy()


def _searchsorted(sorted_a: np.ndarray, v: np.ndarray, right: bool = False) -> np.ndarray:
    """np.searchsorted(sorted_a, v, side="right" if right else "left")."""
    import torch
    return torch.searchsorted(torch.from_numpy(np.ascontiguousarray(sorted_a)),
                              torch.from_numpy(np.ascontiguousarray(v)), right=right).numpy()


def _take(a: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """a[idx] for an integer index array (a gather: one answer)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a))[torch.from_numpy(np.ascontiguousarray(idx))].numpy()


def _sort(a: np.ndarray) -> np.ndarray:
    """np.sort(a)."""
    import torch
    return torch.sort(torch.from_numpy(np.ascontiguousarray(a))).values.numpy()


def _sort_rows(a: np.ndarray) -> np.ndarray:
    """np.sort(a, axis=1) of an integer matrix (integer rows have one sorted order)."""
    import torch
    return torch.sort(torch.from_numpy(np.ascontiguousarray(a)), dim=1).values.numpy()


def _rows_with_repeats(a: np.ndarray) -> np.ndarray:
    """Indices of the rows of a row-sorted matrix that hold a value twice."""
    import torch
    t = torch.from_numpy(a)
    return torch.nonzero((t[:, 1:] == t[:, :-1]).any(dim=1)).reshape(-1).numpy()


def _merge_runs(runs: list) -> np.ndarray:
    """Merge sorted arrays with no value in common into one sorted array
    (numpy's stable sort finds the sorted runs and merges them)."""
    return runs[0] if len(runs) == 1 else np.sort(np.concatenate(runs), kind="stable")


def scaled(spec: dict, factor: float, edges_only: bool = False) -> dict:
    """A workload shape with |U|, |V|, |E| and |A| scaled by factor (the
    attributes per node, exponents, weight laws and seed unchanged): the
    scalability sweep's graphs and the reduced large graph of the tests.
    edges_only scales |E| alone (the sweep by edges: same nodes, sparser)."""
    out = dict(spec)
    if factor != 1.0:
        for key in (("n_e",) if edges_only else ("n_u", "n_v", "n_e", "n_a")):
            out[key] = max(1, int(round(out[key] * factor)))
    return out


def power_law_degrees(rng: np.random.Generator, n: int, gamma: float,
                      total: int, cap: int) -> np.ndarray:
    """Degree sequence of n nodes, Zipf(gamma) shaped, capped, summing to total."""
    if total < n:
        raise ValueError("total degree must be >= number of nodes (d >= 1)")
    if total > n * cap:
        raise ValueError("total degree exceeds n * cap")
    raw = np.minimum(rng.zipf(gamma, size=n), cap).astype(np.float64)
    d = np.floor(raw * (total / raw.sum())).astype(np.int64)
    d = np.clip(d, 1, cap)
    diff = int(total - d.sum())
    guard = 0
    while diff != 0:
        guard += 1
        if guard > 10000:
            raise RuntimeError("degree rescaling did not converge")
        p = d / d.sum()
        if diff > 0:
            d += _choice_counts(rng, p, diff)
            d = np.minimum(d, cap)
        else:
            d -= _choice_counts(rng, p, -diff)
            d = np.maximum(d, 1)
        diff = int(total - d.sum())
    return d


def _unique(a: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + adjacent-difference mask)."""
    a = np.sort(a)
    if a.shape[0] == 0:
        return a
    keep = np.empty(a.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def bipartite_edges(n_u: int, n_v: int, n_e: int, gamma_u: float, gamma_v: float,
                    seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Unique (u, v) pairs, |E| of them, by configuration-model stub matching."""
    if n_e > n_u * n_v:
        raise ValueError("more edges than node pairs")
    du = power_law_degrees(rng_for(seed, _S_DEG_U), n_u, gamma_u, n_e, n_v)
    dv = power_law_degrees(rng_for(seed, _S_DEG_V), n_v, gamma_v, n_e, n_u)
    su = np.repeat(np.arange(n_u, dtype=np.int64), du)
    sv = np.repeat(np.arange(n_v, dtype=np.int64), dv)
    rng_for(seed, _S_PAIR).shuffle(sv)
    # the pair set is kept as sorted runs with no pair in common: the unique
    # stub pairs, then the pairs each top-up round adds
    runs = [_unique(su * n_v + sv)]
    count = runs[0].shape[0]
    rng = rng_for(seed, _S_TOPUP)
    rounds = 0
    while count < n_e:
        rounds += 1
        need = n_e - count
        draw = max(need + need // 2, 1024)
        if rounds <= 16:
            eu = _take(su, rng.integers(0, su.shape[0], size=draw))
            ev = _take(sv, rng.integers(0, sv.shape[0], size=draw))
        else:  # saturated hub pairs: fall back to uniform pairs
            eu = rng.integers(0, n_u, size=draw)
            ev = rng.integers(0, n_v, size=draw)
        cand = eu * n_v + ev
        # keep the first occurrence (in draw order) of every pair not yet
        # present: sort the draws once (stable, so equal pairs keep draw
        # order), test membership with sorted needles, and mark the first of
        # each run of equal pairs
        order = _stable_argsort(cand)
        sc = _take(cand, order)
        keep = np.ones(sc.shape[0], dtype=bool)
        for run in runs:
            pos = _searchsorted(run, sc)
            pos[pos == run.shape[0]] = 0
            keep &= _take(run, pos) != sc
        keep[1:] &= sc[1:] != sc[:-1]
        cand = _take(cand, _sort(order[keep]))[:need]
        runs.append(_sort(cand))
        count += cand.shape[0]
    key = _merge_runs(runs)
    return (key // n_v).astype(np.uint32), (key % n_v).astype(np.uint32)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 value (ties to even): the
    bit pattern b becomes (b + 0x7FFF + bit 16 of b) with the low 16 bits
    cleared, modulo 2^32 (integer arithmetic, on all host cores)."""
    import torch
    b = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32).view(np.int32)).to(torch.int64) & 0xFFFFFFFF
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16) & 0xFFFFFFFF
    b = torch.where(b >= 1 << 31, b - (1 << 32), b).to(torch.int32)
    return b.numpy().view(np.float32)


def node_attributes(n_u: int, n_a: int, m: int, weight_law: str, seed: int,
                    bf16: bool = False, attr_zipf: float | None = None
                    ) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """m distinct attributes per U node with row-normalised positive weights."""
    if m > n_a:
        raise ValueError("m > |A|")
    rng = rng_for(seed, _S_ATTR)
    if attr_zipf is None:
        p = None
    else:
        p = np.arange(1, n_a + 1, dtype=np.float64) ** (-attr_zipf)
        p /= p.sum()

    def draw(rows: int) -> np.ndarray:
        if p is None:
            return rng.integers(0, n_a, size=(rows, m))
        return rng.choice(n_a, size=(rows, m), p=p)

    a = _sort_rows(draw(n_u))
    bad = _rows_with_repeats(a)
    while bad.size:
        a[bad] = _sort_rows(draw(bad.size))
        sub = a[bad]
        bad = bad[_rows_with_repeats(sub)]
    wr = rng_for(seed, _S_AW)
    if weight_law == "uniform":
        w = 1.0 - wr.random(size=(n_u, m))          # uniform(0, 1]
    elif weight_law == "lognormal":
        w = wr.lognormal(0.0, 1.0, size=(n_u, m))
    else:
        raise ValueError(weight_law)
    w = (w / w.sum(axis=1, keepdims=True)).astype(np.float32)
    if bf16:
        w = bf16_round(w)
    w = np.maximum(w, np.float32(np.finfo(np.float32).tiny))  # keep weights > 0
    ea_u = np.repeat(np.arange(n_u, dtype=np.uint32), m)
    return ea_u, a.reshape(-1).astype(np.uint32), w.reshape(-1)


def make_graph(n_u: int, n_v: int, n_e: int, gamma_u: float, gamma_v: float,
               edge_w: str, n_a: int, m: int, attr_w: str, bf16: bool, seed: int,
               attr_zipf: float | None = None) -> GraphArrays:
    """Draw one synthetic attributed bipartite graph (see module docstring)."""
    e_u, e_v = bipartite_edges(n_u, n_v, n_e, gamma_u, gamma_v, seed)
    if edge_w == "unit":
        e_w = np.ones(e_u.shape[0], dtype=np.float32)
    elif edge_w == "uniform_0.5_1.5":
        e_w = (0.5 + rng_for(seed, _S_EW).random(size=e_u.shape[0])).astype(np.float32)
    else:
        raise ValueError(edge_w)
    ea_u, ea_a, ea_w = node_attributes(n_u, n_a, m, attr_w, seed, bf16, attr_zipf)
    meta = dict(n_u=n_u, n_v=n_v, n_e=n_e, gamma_u=gamma_u, gamma_v=gamma_v,
                edge_w=edge_w, n_a=n_a, m=m, attr_w=attr_w, bf16=bf16, seed=seed,
                attr_zipf=attr_zipf)
    return GraphArrays(n_u, n_v, n_a, e_u, e_v, e_w, ea_u, ea_a, ea_w, meta)


def draw_queries(n_u: int, count: int, seed: int = 11, stream: int = _S_QUERY) -> np.ndarray:
    """count query nodes drawn uniformly from U (with replacement)."""
    return rng_for(seed, stream).integers(0, n_u, size=count).astype(np.uint32)


def draw_stream(count: int, rate_qps: float, n_u: int, seed: int = 101,
                eps_lo: float = 1e-7, eps_hi: float = 1e-4,
                ks: tuple[int, ...] = (10, 100, 1000)):
    """Open-loop Poisson request stream: arrival times (s), nodes, eps, k.

    eps is log-uniform in [eps_lo, eps_hi]; k is uniform over ks.
    """
    r = rng_for(seed, 0)
    gaps = r.exponential(1.0 / rate_qps, size=count)
    t = np.cumsum(gaps) - gaps[0]
    q = rng_for(seed, 1).integers(0, n_u, size=count).astype(np.uint32)
    le = rng_for(seed, 2).uniform(np.log(eps_lo), np.log(eps_hi), size=count)
    k = np.asarray(ks, dtype=np.uint32)[rng_for(seed, 3).integers(0, len(ks), size=count)]
    return t, q, np.exp(le), k
