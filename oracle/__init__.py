"""CPU oracle for approximate single-source AHPP queries.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (no kernels, headers, helpers or constants) and never
imports it; both sides receive the same seeded COO arrays.

Two layers:
  * the C library ``ahpp_oracle.c`` (FP64, one thread): the two-hop
    x -> xP of Eq. 1 / Eq. 2, Power Iteration (Algorithm 1), the lambda
    estimate (Theorem 3), Forward Push (Algorithm 2), APP (Algorithm 3) and
    ASRP (Algorithm 4) with per-round traces, and a plain top-k;
  * numpy code for tiny graphs only: the dense P_S of Eq. 1 and P_A of
    Eq. 2 written from their definitions, exact AHPP by a dense linear solve
    of Def. 2 / Eq. 3, the full similarity matrix Pi (for Lemma 3 and
    Theorem 3 checks), and a Monte Carlo simulation of the random walk of
    Lemma 1.

Parity status: every function here is pinned by the tests in
``tests/test_oracle_*.py`` (worked example of Section 2.1, closed forms,
Lemma 1 sampling, Lemma 3 per round, Theorems 2 and 3).  The ASRP switch
test of Algorithm 4 is printed in a garbled form; the oracle implements the
reading that Theorem 1's proof supports (and the printed form as an
option), and both are pinned by the trajectory worked out by hand on a
graph with P = J/n (switch round, rounds, pushed entries, traces, reserves)
and by the selection rule of each phase on a power-law graph.  No printed
trajectory exists to pin the reading itself against.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

OG_FP, OG_APP, OG_ASRP, OG_APPS = 0, 1, 2, 3
ALGOS = {"fp": OG_FP, "app": OG_APP, "asrp": OG_ASRP, "apps": OG_APPS}

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


class _Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("switch_round", ctypes.c_uint32),
                ("n_p", ctypes.c_uint64), ("pushes", ctypes.c_uint64),
                ("resid_sum", ctypes.c_double), ("reserve_sum", ctypes.c_double),
                ("leak", ctypes.c_double), ("max_resid", ctypes.c_double)]


class _PushState(ctypes.Structure):
    """Where a resumable push stands between rounds (og_push_state)."""
    _fields_ = [("round", ctypes.c_uint32), ("sync", ctypes.c_uint32),
                ("switch_round", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("n_p", ctypes.c_uint64), ("pushes", ctypes.c_uint64), ("leak", ctypes.c_double)]


class _Trace(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_uint32), ("frontier", _u64p), ("n_p", _u64p),
                ("max_r", _f64p), ("sum_r", _f64p), ("sum_pi", _f64p), ("phase", _u8p)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle())
        L.og_build.restype = ctypes.c_void_p
        L.og_build.argtypes = [ctypes.c_uint32] * 3 + [ctypes.c_uint64, _u32p, _u32p, _f64p,
                                                       ctypes.c_uint64, _u32p, _u32p, _f64p]
        L.og_free.argtypes = [ctypes.c_void_p]
        L.og_num_edges.restype = ctypes.c_uint64
        L.og_num_edges.argtypes = [ctypes.c_void_p]
        L.og_num_attr_edges.restype = ctypes.c_uint64
        L.og_num_attr_edges.argtypes = [ctypes.c_void_p]
        L.og_node_stats.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p, _f64p, _u32p]
        L.og_power_iteration.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_uint32, ctypes.c_uint32, _f64p]
        L.og_lambda.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                ctypes.c_uint32, _f64p, _f64p]
        L.og_push.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                              ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                              ctypes.c_uint32, _f64p, _f64p, ctypes.POINTER(_Stats),
                              ctypes.POINTER(_Trace)]
        L.og_push_start.argtypes = [ctypes.c_void_p, ctypes.c_uint32, _f64p, _f64p,
                                    ctypes.POINTER(_PushState)]
        L.og_push_resume.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint32,
                                     _f64p, _f64p, ctypes.POINTER(_PushState), ctypes.POINTER(_Stats)]
        L.og_forward_push.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64,
                                      _f64p, _f64p, ctypes.POINTER(_Stats)]
        L.og_topk.argtypes = [_f64p, ctypes.c_uint32, ctypes.c_uint32, _u32p, _f64p]
        _lib = L
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def default_lambda_T(n_u: int, alpha: float) -> int:
    """Iterations of the Theorem 3 estimate: the tail |U|(1-alpha)^T <= 0.01."""
    return int(math.ceil(math.log(100.0 * max(n_u, 1)) / math.log(1.0 / (1.0 - alpha))))


@dataclass
class PushResult:
    pi: np.ndarray          # reserves pi_hat(q, .) over U
    r_u: np.ndarray         # residues r(q, .) over U at exit
    rc: int                 # 0 converged, 1 round cap reached
    stats: dict
    trace: dict


class OracleGraph:
    """The oracle's own copy of G, built from COO arrays (weights in FP64)."""

    def __init__(self, n_u, n_v, n_a, e_u, e_v, e_w, ea_u, ea_a, ea_w):
        self.n_u, self.n_v, self.n_a = int(n_u), int(n_v), int(n_a)
        e_u = np.ascontiguousarray(e_u, dtype=np.uint32)
        e_v = np.ascontiguousarray(e_v, dtype=np.uint32)
        e_w = np.ascontiguousarray(e_w, dtype=np.float64)
        ea_u = np.ascontiguousarray(ea_u, dtype=np.uint32)
        ea_a = np.ascontiguousarray(ea_a, dtype=np.uint32)
        ea_w = np.ascontiguousarray(ea_w, dtype=np.float64)
        h = lib().og_build(self.n_u, self.n_v, self.n_a,
                           e_u.shape[0], _p(e_u, _u32p), _p(e_v, _u32p), _p(e_w, _f64p),
                           ea_u.shape[0], _p(ea_u, _u32p), _p(ea_a, _u32p), _p(ea_w, _f64p))
        if not h:
            raise ValueError("oracle: invalid graph (index out of range or weight <= 0)")
        self._h = ctypes.c_void_p(h)

    @classmethod
    def from_arrays(cls, g) -> "OracleGraph":
        return cls(g.n_u, g.n_v, g.n_a, g.e_u, g.e_v, g.e_w, g.ea_u, g.ea_a, g.ea_w)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.og_free(h)
            self._h = None

    @property
    def n_e(self) -> int:
        return int(lib().og_num_edges(self._h))

    @property
    def n_ea(self) -> int:
        return int(lib().og_num_attr_edges(self._h))

    def node_stats(self) -> dict:
        d_u = np.zeros(self.n_u); d_v = np.zeros(self.n_v)
        wr = np.zeros(self.n_u); wc = np.zeros(self.n_a)
        cnt = np.zeros(self.n_u, dtype=np.uint32)
        lib().og_node_stats(self._h, _p(d_u, _f64p), _p(d_v, _f64p), _p(wr, _f64p),
                            _p(wc, _f64p), _p(cnt, _u32p))
        return dict(d_u=d_u, d_v=d_v, wrow_u=wr, wcol_a=wc, cnt_u=cnt)

    def power_iteration(self, alpha: float, beta: float, q: int, T: int) -> np.ndarray:
        """Algorithm 1; absolute error <= (1 - alpha)^T."""
        pi = np.zeros(self.n_u)
        rc = lib().og_power_iteration(self._h, alpha, beta, q, T, _p(pi, _f64p))
        if rc != 0:
            raise ValueError(f"oracle power iteration failed ({rc})")
        return pi

    def lambda_estimate(self, alpha: float, beta: float, T: int | None = None):
        """Theorem 3: (lambda, pi_T)."""
        if T is None:
            T = default_lambda_T(self.n_u, alpha)
        lam = ctypes.c_double(0.0)
        piT = np.zeros(self.n_u)
        rc = lib().og_lambda(self._h, alpha, beta, T, ctypes.byref(lam), _p(piT, _f64p))
        if rc != 0:
            raise ValueError(f"oracle lambda failed ({rc})")
        return lam.value, piT

    def push(self, algo: str, alpha: float, beta: float, q: int, eps: float,
             lam: float | None = None, switch_rule: int = 0, max_rounds: int = 1_000_000,
             trace_cap: int = 4096) -> PushResult:
        """APP (Algorithm 3), ASRP (Algorithm 4) or APP(S) (APP with ASRP's
        synchronous switch, the ablation arm of Exp-2) from q."""
        pi = np.zeros(self.n_u)
        r_u = np.zeros(self.n_u)
        st = _Stats()
        cap = max(1, min(trace_cap, max_rounds))
        buf = dict(frontier=np.zeros(cap, np.uint64), n_p=np.zeros(cap, np.uint64),
                   max_r=np.zeros(cap), sum_r=np.zeros(cap), sum_pi=np.zeros(cap),
                   phase=np.zeros(cap, np.uint8))
        tr = _Trace(cap, _p(buf["frontier"], _u64p), _p(buf["n_p"], _u64p),
                    _p(buf["max_r"], _f64p), _p(buf["sum_r"], _f64p),
                    _p(buf["sum_pi"], _f64p), _p(buf["phase"], _u8p))
        rc = lib().og_push(self._h, ALGOS[algo], alpha, beta, q, eps,
                           0.0 if lam is None else float(lam), switch_rule, max_rounds,
                           _p(pi, _f64p), _p(r_u, _f64p), ctypes.byref(st), ctypes.byref(tr))
        if rc < 0:
            raise ValueError(f"oracle push failed ({rc})")
        stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
        n = min(stats["rounds"], cap)
        trace = {k: v[:n].copy() for k, v in buf.items()}
        return PushResult(pi, r_u, rc, stats, trace)

    def push_start(self, q: int) -> "ResumablePush":
        """The initial state of a push from q (unit residue at q), to be
        advanced by push_resume a few rounds at a time."""
        r = ResumablePush(np.zeros(self.n_u), np.zeros(self.n_u), _PushState())
        rc = lib().og_push_start(self._h, q, _p(r.pi, _f64p), _p(r.r_u, _f64p), ctypes.byref(r.state))
        if rc < 0:
            raise ValueError(f"oracle push start failed ({rc})")
        return r

    def push_resume(self, r: "ResumablePush", algo: str, alpha: float, beta: float, eps: float,
                    lam: float | None = None, switch_rule: int = 0, rounds: int = 1) -> int:
        """At most `rounds` more rounds of the push in r (updated in place);
        returns 0 once converged, 1 if rounds ran out first.  Its stats hold
        the totals so far."""
        st = _Stats()
        rc = lib().og_push_resume(self._h, ALGOS[algo], alpha, beta, eps,
                                  0.0 if lam is None else float(lam), switch_rule, rounds,
                                  _p(r.pi, _f64p), _p(r.r_u, _f64p), ctypes.byref(r.state),
                                  ctypes.byref(st))
        if rc < 0:
            raise ValueError(f"oracle push resume failed ({rc})")
        r.stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
        return rc

    def forward_push(self, alpha: float, beta: float, q: int, eps: float,
                     max_pushes: int = 1 << 40) -> PushResult:
        """Algorithm 2 (FIFO order)."""
        pi = np.zeros(self.n_u)
        r_u = np.zeros(self.n_u)
        st = _Stats()
        rc = lib().og_forward_push(self._h, alpha, beta, q, eps, max_pushes,
                                   _p(pi, _f64p), _p(r_u, _f64p), ctypes.byref(st))
        if rc < 0:
            raise ValueError(f"oracle forward push failed ({rc})")
        stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
        return PushResult(pi, r_u, rc, stats, {})


@dataclass
class ResumablePush:
    """Reserves, residues and round state of a push advanced in pieces."""
    pi: np.ndarray
    r_u: np.ndarray
    state: _PushState
    stats: dict | None = None


def topk(score: np.ndarray, k: int):
    """k largest scores; score descending, node id ascending on ties."""
    score = np.ascontiguousarray(score, dtype=np.float64)
    k = min(int(k), score.shape[0])
    nodes = np.zeros(k, np.uint32)
    vals = np.zeros(k)
    n = lib().og_topk(_p(score, _f64p), score.shape[0], k, _p(nodes, _u32p), _p(vals, _f64p))
    return nodes[:n], vals[:n]


# --------------------------------------------------------------- dense (tiny)

def dense_matrices(n_u, n_v, n_a, e_u, e_v, e_w, ea_u, ea_a, ea_w, beta):
    """P_S (Eq. 1), P_A (Eq. 2) and P = (1-beta) P_S + beta P_A, dense FP64.

    Rows of a node without V neighbours (attributes) are zero in P_S (P_A).
    """
    W = np.zeros((n_u, n_v))
    np.add.at(W, (np.asarray(e_u, np.int64), np.asarray(e_v, np.int64)),
              np.asarray(e_w, np.float64))
    WA = np.zeros((n_u, n_a))
    np.add.at(WA, (np.asarray(ea_u, np.int64), np.asarray(ea_a, np.int64)),
              np.asarray(ea_w, np.float64))
    d_u = W.sum(axis=1)
    d_v = W.sum(axis=0)
    row_a = WA.sum(axis=1)
    col_a = WA.sum(axis=0)
    # P_S[i, j] = sum_v w(i, v) / d(i) * w(v, j) / d(v)
    left = np.divide(W, d_u[:, None], out=np.zeros_like(W), where=d_u[:, None] > 0)
    right = np.divide(W, d_v[None, :], out=np.zeros_like(W), where=d_v[None, :] > 0)
    P_S = left @ right.T
    # P_A[i, j] = sum_a w(i, a) / sum_a' w(i, a') * w(j, a) / sum_k w(k, a)
    leftA = np.divide(WA, row_a[:, None], out=np.zeros_like(WA), where=row_a[:, None] > 0)
    rightA = np.divide(WA, col_a[None, :], out=np.zeros_like(WA), where=col_a[None, :] > 0)
    P_A = leftA @ rightA.T
    return P_S, P_A, (1.0 - beta) * P_S + beta * P_A


def dense_matrices_of(g, beta):
    return dense_matrices(g.n_u, g.n_v, g.n_a, g.e_u, g.e_v, g.e_w, g.ea_u, g.ea_a,
                          g.ea_w, beta)


def exact_dense(P: np.ndarray, alpha: float, q: int) -> np.ndarray:
    """pi(q, .) of Eq. 3 summed in closed form: x (I - (1-alpha) P) = alpha e_q."""
    n = P.shape[0]
    rhs = np.zeros(n)
    rhs[q] = alpha
    return np.linalg.solve((np.eye(n) - (1.0 - alpha) * P).T, rhs)


def pi_matrix(P: np.ndarray, alpha: float) -> np.ndarray:
    """Pi[i, j] = pi(u_i, u_j) = alpha [(I - (1-alpha) P)^-1]_{ij}."""
    n = P.shape[0]
    return alpha * np.linalg.inv(np.eye(n) - (1.0 - alpha) * P)


def series_sum(P: np.ndarray, alpha: float, q: int, terms: int) -> np.ndarray:
    """Eq. 3 truncated: sum_{l < terms} alpha (1-alpha)^l P^l[q, .]."""
    x = np.zeros(P.shape[0])
    x[q] = 1.0
    out = np.zeros_like(x)
    for l in range(terms):
        out += alpha * (1.0 - alpha) ** l * x
        x = x @ P
    return out


def monte_carlo_walks(g, alpha: float, beta: float, q: int, n_walks: int,
                      seed: int = 7, max_steps: int = 10_000) -> np.ndarray:
    """Empirical stop distribution of the walk of Lemma 1 from q.

    Each step: stop with probability alpha; otherwise with probability
    1 - beta take a structure move (v with prob. w(u,v)/d(u), then u' with
    prob. w(v,u')/d(v)) and with probability beta an attribute move (a with
    prob. w(u,a)/sum_a' w(u,a'), then u' with prob. w(u',a)/sum_k w(k,a)).
    A walk that must move from a node without the chosen kind of neighbour
    is lost (it counts nowhere).
    """
    rng = np.random.Generator(np.random.Philox(key=np.array([seed, 99], np.uint64)))

    def csr(rows, cols, w, n_rows):
        rows = np.asarray(rows, np.int64)
        order = np.argsort(rows, kind="stable")
        cols = np.asarray(cols, np.int64)[order]
        w = np.asarray(w, np.float64)[order]
        off = np.zeros(n_rows + 1, np.int64)
        np.add.at(off, rows + 1, 1)
        off = np.cumsum(off)
        cum = np.cumsum(w)
        start = np.concatenate([[0.0], cum])[off[:-1]]
        total = np.concatenate([[0.0], cum])[off[1:]] - start
        return off, cols, cum, start, total

    UV = csr(g.e_u, g.e_v, g.e_w, g.n_u)
    VU = csr(g.e_v, g.e_u, g.e_w, g.n_v)
    UA = csr(g.ea_u, g.ea_a, g.ea_w, g.n_u)
    AU = csr(g.ea_a, g.ea_u, g.ea_w, g.n_a)

    def hop(adj, src):
        off, cols, cum, start, total = adj
        ok = total[src] > 0
        t = start[src] + rng.random(src.shape[0]) * total[src]
        idx = np.searchsorted(cum, t, side="right")
        idx = np.minimum(np.maximum(idx, off[src]), np.maximum(off[src + 1] - 1, 0))
        return np.where(ok, cols[np.minimum(idx, cols.shape[0] - 1)], -1)

    counts = np.zeros(g.n_u)
    pos = np.full(n_walks, q, np.int64)
    for _ in range(max_steps):
        if pos.shape[0] == 0:
            break
        stop = rng.random(pos.shape[0]) < alpha
        np.add.at(counts, pos[stop], 1.0)
        pos = pos[~stop]
        attr = rng.random(pos.shape[0]) < beta
        nxt = np.empty_like(pos)
        s = pos[~attr]
        mid = hop(UV, s)
        okm = mid >= 0
        out = np.full(s.shape[0], -1, np.int64)
        out[okm] = hop(VU, mid[okm])
        nxt[~attr] = out
        s = pos[attr]
        mid = hop(UA, s)
        okm = mid >= 0
        out = np.full(s.shape[0], -1, np.int64)
        out[okm] = hop(AU, mid[okm])
        nxt[attr] = out
        pos = nxt[nxt >= 0]
    return counts / n_walks
