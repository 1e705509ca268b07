"""FP64 oracle runs in worker processes (test infrastructure).

The full-size parity tests need several oracle pushes and exact Power
Iterations on graphs with 10^7-10^8 edges; each takes up to minutes on one
core, so they run in parallel worker processes.  Workers are started with
the spawn method (a process forked after the parent has used the GPU may
hang) and rebuild the graph from its seeded recipe (synth), so no graph
arrays are pickled.  Start the jobs before the GPU work of a test and
collect them after it: the two overlap.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os

_OG = None


def _init(spec: dict) -> None:
    global _OG
    import oracle
    from paper_2512_11606_gb300 import synth
    _OG = oracle.OracleGraph.from_arrays(synth.make_graph(**spec))


def _run(job: tuple):
    kind = job[0]
    if kind == "push":                 # ("push", algo, alpha, beta, q, eps, lam, switch_rule)
        _, algo, alpha, beta, q, eps, lam, rule = job
        r = _OG.push(algo, alpha, beta, q, eps, lam=lam, switch_rule=rule)
        return r.pi, dict(r.stats)
    if kind == "pi":                   # ("pi", alpha, beta, q, T): Algorithm 1's T-th iterate
        _, alpha, beta, q, T = job
        return _OG.power_iteration(alpha, beta, q, T), {"T": T}
    raise ValueError(kind)


def exact_T(alpha: float, tail: float = 1e-10) -> int:
    """Iterations of Algorithm 1 after which (1 - alpha)^T <= tail: the
    iterate is then within tail of exact AHPP (Eq. 3) in every entry."""
    return int(math.ceil(math.log(tail) / math.log(1.0 - alpha)))


class Jobs:
    """Oracle jobs on one graph recipe, running in the background."""

    def __init__(self, spec: dict, jobs: list, processes: int | None = None):
        n = processes or max(1, min(len(jobs), os.cpu_count() or 1))
        self._pool = mp.get_context("spawn").Pool(n, initializer=_init, initargs=(dict(spec),))
        self._res = self._pool.map_async(_run, list(jobs), chunksize=1)

    def get(self, timeout: float = 1800.0) -> list:
        try:
            return self._res.get(timeout)
        finally:
            self._pool.close()
            self._pool.join()

    def cancel(self) -> None:
        self._pool.terminate()
        self._pool.join()


def push_job(q, eps, lam, algo="asrp", alpha=0.15, beta=0.35, switch_rule=0) -> tuple:
    return ("push", algo, alpha, beta, int(q), float(eps), float(lam), int(switch_rule))


def pi_job(q, T, alpha=0.15, beta=0.35) -> tuple:
    return ("pi", alpha, beta, int(q), int(T))
