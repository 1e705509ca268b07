#!/usr/bin/env python
"""AHPP query throughput on one GB300 (or N, one process per GPU).

Workload (default): the medium synthetic attributed bipartite graph
(|U| = 1M, |V| = 500k, |E| = 20M Zipf(2.1) degrees, uniform(0.5,1.5) FP32
edge weights; |A| = 10k attributes, 20 per node, lognormal weights,
row-normalised, stored as bfloat16), ASRP with the Theorem 3 lambda,
eps = 1e-6, top-100.  One step = one batch of 1,024 queries drawn uniformly
from U, pushed by the batched persistent launch (graph and query arrays
resident in HBM).  The plain one-query-at-a-time GPU push is timed on the
same graph as the comparison point, and the FP64 CPU oracle on the host
cores as the CPU baseline.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead (the reference arm; this paper has no reference code), in bounded
steps: one query in flight per host core, each step advancing them a few
rounds from their kept state.
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2512_11606_gb300 import synth  # noqa: E402  (input recipe only)

ALPHA, BETA = 0.15, 0.35
METRIC = "AHPP queries/sec at eps=1e-6 (batched persistent push)"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--k", type=int, default=100)
    ap.add_argument("--plain-queries", type=int, default=6)
    ap.add_argument("--cpu-queries", type=int, default=0, help="0: one per host core (max 16)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--graph", default="medium", choices=["medium", "tiny", "large"])
    ap.add_argument("--scale", type=float, default=1.0,
                    help="large graph only: scale |U|, |V|, |E| and |A| by this factor (scalability sweep)")
    ap.add_argument("--scale-edges-only", action="store_true",
                    help="with --scale: scale |E| alone (the sweep by edges; nodes unchanged)")
    ap.add_argument("--ablation", type=int, default=3,
                    help="single-query ablation of the ASRP switch rule and APP on N queries (0: off)")
    ap.add_argument("--scale-leg", type=float, default=0.25,
                    help="also time batched and plain queries on the large recipe scaled by this factor "
                         "(the scalability sweep's smallest graph; 0: off)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (no ahpp_autotune before the timed region)")
    ap.add_argument("--no-exact", action="store_true",
                    help="skip the exact AHPP references (oracle Algorithm 1) of the parity leg")
    ap.add_argument("--cost-queries", type=int, default=4,
                    help="queries whose bfloat16 precision cost is measured (exact AHPP, two graphs)")
    ap.add_argument("--serve-seconds", type=float, default=12.0,
                    help="open-loop serving window (0 disables the serving measurement)")
    ap.add_argument("--serve-load", type=float, default=0.8,
                    help="Poisson arrival rate as a fraction of the measured batched capacity")
    ap.add_argument("--serve-slots", type=int, default=32)
    ap.add_argument("--serve-rounds", type=int, default=4)
    ap.add_argument("--ref-step-seconds", type=float, default=5.0,
                    help="reference arm: target wall time of one bounded step (a few rounds of each query in flight)")
    return ap.parse_args(argv)


def graph_spec(name, scale=1.0, edges_only=False):
    if name == "large":
        return synth.scaled(synth.LARGE, scale, edges_only)
    return dict(synth.MEDIUM_BF16) if name == "medium" else dict(synth.TINY, bf16=True)


def workload_config(args, extra=None):
    spec = graph_spec(args.graph, args.scale, args.scale_edges_only)
    cfg = {
        "workload": (f"{args.graph} attributed bipartite graph |U|={spec['n_u']:,} |V|={spec['n_v']:,} "
                     f"|E|={spec['n_e']:,} Zipf({spec['gamma_u']}) degrees, |A|={spec['n_a']:,} "
                     f"x{spec['m']} bf16 attribute weights; ASRP (Theorem 3 lambda), "
                     f"alpha={ALPHA}, beta={BETA}, eps={args.eps:g}, top-{args.k}; "
                     f"{args.batch} queries per step (batched persistent launch)"),
        "graph": (args.graph if args.scale == 1.0 else
                  f"{args.graph} x{args.scale:g}{' edges only' if args.scale_edges_only else ''}"),
        "batch_queries_per_gpu": args.batch,
        "eps": args.eps,
        "k": args.k,
        "l2": ("inputs larger than L2 (graph ~0.7 GB + per-tile state ~0.45 GB per round)"
               if args.graph == "medium" else
               "inputs larger than L2 (graph ~5 GB + per-tile state ~2.3 GB per round)"
               if args.graph == "large" else "tiny graph: L2-resident, reported, not graded"),
        "parallelism": f"replicas{args.gpus}" if args.gpus > 1 else "1 GPU",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------- oracle

_OG = None


def _oracle_worker(args):
    q, eps, lam = args
    t0 = time.perf_counter()
    res = _OG.push("asrp", ALPHA, BETA, int(q), eps, lam=lam)
    return time.perf_counter() - t0, res.stats["rounds"]


def _ref_core(conn, queries, eps, lam):
    """One host core of the reference arm: keeps one oracle ASRP query in
    flight and, per command, advances it by a number of rounds from its kept
    state (starting the next query whenever one converges).  Replies with the
    wall time, the rounds run and the round counts of the queries that
    converged."""
    it = itertools.cycle(queries)
    cur = None
    while True:
        budget = conn.recv()
        if budget is None:
            break
        t0 = time.perf_counter()
        ran, finished = 0, []
        while ran < budget:
            if cur is None:
                cur = _OG.push_start(int(next(it)))
            before = cur.state.round
            rc = _OG.push_resume(cur, "asrp", ALPHA, BETA, eps, lam=lam, rounds=budget - ran)
            ran += cur.state.round - before
            if rc == 0:
                finished.append(cur.state.round)
                cur = None
        conn.send((time.perf_counter() - t0, ran, finished))
    conn.close()


def _oracle_worker_pi(args):
    """As _oracle_worker, also returning the reserve vector (for parity)."""
    q, eps, lam = args
    t0 = time.perf_counter()
    res = _OG.push("asrp", ALPHA, BETA, int(q), eps, lam=lam)
    return time.perf_counter() - t0, res.stats["rounds"], res.pi


def cpu_oracle_sample(g, eps, n_queries, seed=11):
    """Time the FP64 oracle (as it stands) on a bounded sample of queries,
    one query per process (fork before any CUDA use)."""
    import oracle
    global _OG
    t0 = time.perf_counter()
    _OG = oracle.OracleGraph.from_arrays(g)
    lam, _ = _OG.lambda_estimate(ALPHA, BETA)
    prep = time.perf_counter() - t0
    qs = synth.draw_queries(g.n_u, n_queries, seed=seed)
    ctx = mp.get_context("fork")
    t1 = time.perf_counter()
    with ctx.Pool(n_queries) as pool:
        out = pool.map(_oracle_worker_pi, [(int(q), eps, lam) for q in qs])
    wall = time.perf_counter() - t1
    lat = [o[0] for o in out]
    return {
        "value": n_queries / wall,
        "unit": "queries/s",
        "cores": n_queries,
        "cpu_model": host_cpu_model(),
        "kind": "oracle",
        "sample": (f"{n_queries} ASRP queries (FP64, single-threaded each, one process per core) "
                   f"on the same graph; wall {wall:.1f} s; per-query p50 "
                   f"{statistics.median(lat) * 1e3:.0f} ms; oracle lambda {lam:.2f} computed in "
                   f"{prep:.1f} s preprocessing (not timed)"),
        "lambda": lam,
        "queries": [int(q) for q in qs],
        "pi": [o[2] for o in out],
        "p50_ms": statistics.median(lat) * 1e3,
        "p99_ms": float(np.percentile(lat, 99)) * 1e3,
    }


# Exact AHPP references (Algorithm 1 until (1 - alpha)^T <= 1e-10, FP64 oracle),
# run in a pool forked before any CUDA use and collected after the GPU legs.
_OG32 = None
EXACT_TAIL = 1e-10


def exact_T(alpha=ALPHA, tail=EXACT_TAIL):
    return int(math.ceil(math.log(tail) / math.log(1.0 - alpha)))


def _exact_worker(args):
    which, q, T = args
    og = _OG if which == "graph" else _OG32
    return og.power_iteration(ALPHA, BETA, int(q), T)


def start_exact_refs(g, spec, cpu, n_cost, processes):
    """Start the oracle's exact AHPP of the CPU-baseline sample queries (on
    the benchmarked graph) and, for the first n_cost of them, on the same
    graph with its attribute weights left in FP32 (not rounded to bfloat16):
    the precision cost of storing them as bfloat16 (reading C-7).  Forks its
    workers now (call before CUDA is initialised); returns (pool, async
    result, job list)."""
    import oracle
    global _OG32
    jobs = [("graph", int(q), exact_T()) for q in cpu["queries"]]
    if spec.get("bf16") and n_cost > 0:
        g32 = synth.make_graph(**dict(spec, bf16=False))
        _OG32 = oracle.OracleGraph.from_arrays(g32)
        jobs += [("fp32", int(q), exact_T()) for q in cpu["queries"][:n_cost]]
    pool = mp.get_context("fork").Pool(max(1, min(processes, len(jobs))))
    return pool, pool.map_async(_exact_worker, jobs, chunksize=1), jobs


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def host_cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


# ------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


def measured_peak():
    """HBM peak (GB/s) and where it came from: the measured copy bandwidth of
    MEASURED_PEAKS.json, else the profiling recipe's fallback of 6.8 TB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured hbm_gbs (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


# ------------------------------------------------------------ byte model

def round_bytes(info, lanes, bf16=True):
    """Algorithmic DRAM bytes of one pull round of a tile with `lanes` queries.

    Graph (once per round, shared by the lanes): phase 1 streams V->U (index
    + coefficient, 8 B/edge); phase 2 streams U->V (index + weight, 8 B/edge)
    and U->A (index + bf16 weight for the gather, FP32 push coefficient for the
    attribute push: 10 B/entry; the push re-reads the index the gather read);
    row offsets of the three directions.  State (per lane): phase 1 reads r_U
    once, writes t_V, scans t_A and clears the next t_A; phase 2 reads t_V and
    t_A once, reads and writes r_U, and read-modify-writes the reserve and its
    Kahan compensation.
    """
    wa = 2 if bf16 else 4
    nU, nV, nA, nE, nEA = (info[k] for k in ("n_u", "n_v", "n_a", "n_e", "n_ea"))
    graph = 2 * (4 + 4) * nE + (4 + wa + 4) * nEA + 4 * (2 * (nU + 1) + nV + 1)
    state = lanes * 4 * (nU + nV + 2 * nA + nV + nA + 2 * nU + 4 * nU)
    return graph + state


def q1_round_bytes(info, bf16=True):
    """Algorithmic DRAM bytes of one pull round of the single-query kernel.

    Graph (once per round): phase 1 streams V->U (index + coefficient,
    8 B/edge); phase 2 streams U->V (index + weight, 8 B/edge) and U->A
    (index + weight, 4 + 2 B/entry in bfloat16); the row offsets; the
    attribute normalisers.  With the attribute push (single_attr_push) the
    attribute hop reuses phase 2's U->A stream; without it phase 1 also
    streams A->U (index + FP32 pull coefficient, 8 B/entry).  State: the
    residues gathered in phase 1 (each read once), t_V written and read,
    t_A read, written (or pushed) and cleared, the residues read and written,
    the reserve and its Kahan compensation read and written.
    """
    wa = 2 if bf16 else 4
    nU, nV, nA, nE, nEA = (info[k] for k in ("n_u", "n_v", "n_a", "n_e", "n_ea"))
    graph = 2 * 8 * nE + (4 + wa) * nEA + 4 * (2 * (nU + 1) + (nV + 1)) + 4 * (nU + nA)
    if not info.get("single_attr_push", 0):
        graph += 8 * nEA + 4 * (nA + 1)
    state = 4 * (nU + 2 * nV + 3 * nA + 2 * nU + 4 * nU)
    return graph + state


def decode_stats(ahpp, raw):
    """ahpp_stats records from a [n, sizeof(ahpp_stats)] byte tensor."""
    ctype_to_np = {"c_uint": "u4", "c_ulong": "u8", "c_double": "f8", "c_int": "i4"}
    return np.frombuffer(raw.cpu().numpy().view(np.uint8).tobytes(), dtype=np.dtype(
        [(f.rstrip("_"), ctype_to_np[t.__name__]) for f, t in ahpp.Stats._fields_]))


def topk_bytes(info, queries):
    return queries * 4 * info["n_u"]


# DRAM and L2 -> SM bytes of the two push kernels on the medium graph, from
# ncu captures summarised under profiles/ (k_tiles: one 32-query tile, per
# tile-round; k_query1: one query, per pull round).  Each figure describes
# the kernel built from the sources listed by code digest; once the code of
# any of them changes (comments and layout aside) the figure no longer
# applies and ncu_traffic returns None.
NCU_TRAFFIC = {
    # ncu --set full of one 32-query tile on the medium graph (106 tile-rounds):
    # profiles/k_tiles_medium_tile32.md
    "k_tiles": {
        "graph": "medium",
        "bytes_per_unit": 2.424642e9,        # dram__bytes_read.sum + dram__bytes_write.sum per tile-round
        "l2_to_sm_bytes_per_unit": 8.972795e9,   # l1tex__m_xbar2l1tex_read_bytes.sum per tile-round
        "sources": {"ahpp_batch_kernel.cuh": "f341ce418086809a", "ahpp_batch.cu": "f92167d838a2d532",
                    "ahpp_batch.cuh": "2f7f8c2bb4bfbcdd", "ahpp_internal.cuh": "45194dba8b4be444"},
    },
    # the same capture's third k_query1 launch, one plain query (105 pull rounds):
    # profiles/k_query1_medium.md
    "k_query1": {
        "graph": "medium",
        "bytes_per_unit": 5.008213e8,        # per pull round
        "l2_to_sm_bytes_per_unit": 1.402732e9,
        "sources": {"ahpp_query1.cu": "90fefeb4b00d7cd3", "ahpp_query1.cuh": "e356ae0e412d9385",
                    "ahpp_internal.cuh": "45194dba8b4be444"},
    },
}


def code_digest(text):
    """sha256 prefix of C/C++/CUDA source with its comments removed and every
    run of whitespace made one space: the same for two versions of a file
    that differ only in comments or layout, different when the code differs."""
    import hashlib
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":                                  # string or character literal
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    code = " ".join("".join(out).split())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def ncu_traffic(kernel, graph, units, key="bytes_per_unit"):
    """Bytes of one launch scaled from the capture of `kernel` (DRAM by
    default, or the L2 -> SM bytes) by its units (tile-rounds or pull
    rounds), or None if no capture describes the kernel as built now (the
    code of a source file, comments aside, differs from the captured)."""
    rec = NCU_TRAFFIC[kernel]
    if graph != rec["graph"] or rec[key] is None or not rec["sources"]:
        return None
    csrc = os.path.join(ROOT, "paper_2512_11606_gb300", "csrc")
    for name, want in rec["sources"].items():
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            if code_digest(f.read()) != want:
                return None
    return rec[key] * units


def row_roofline(ahpp, info, tile_rounds, launch_s, device):
    """The batched launch against the L2 row-access ceiling of this GPU.

    Per tile-round the kernel gathers |E| residue rows (phase 1, from the
    tile's |U| x 128-byte residue table), |E| t_V rows and |E_A| t_A rows
    (phase 2), and reduces |E_A| rows into the next round's t_A (the attribute
    push).  The ceiling is the time those row accesses take at the rates
    ahpp_row_access_peak measures for tables of the same sizes; frac is that
    time over the measured launch time (the streamed graph and state bytes
    are left out of the ceiling, so frac is an upper estimate of the gap).
    """
    nU, nV, nA, nE, nEA = (int(info[k]) for k in ("n_u", "n_v", "n_a", "n_e", "n_ea"))
    row = 4 * int(info["batch_tile"])
    parts = [("gather", nU * row, nE, "phase 1: residue rows"),
             ("gather", nV * row, nE, "phase 2: t_V rows"),
             ("gather", nA * row, nEA, "phase 2: t_A rows"),
             ("reduce", nA * row, nEA, "phase 2: attribute push into t_A")]
    rates, t_min = [], 0.0
    for op, table, n, what in parts:
        r = ahpp.row_access_peak(table, op, device)
        rates.append({"what": what, "op": op, "table_bytes": table, "rows_per_tile_round": n,
                      "peak_rows_per_s": r})
        t_min += n / r
    rows = tile_rounds * sum(p[2] for p in parts)
    return {"bound": "l2 row access", "unit": "rows/s",
            "achieved": rows / launch_s, "peak": rows / (tile_rounds * t_min),
            "frac": tile_rounds * t_min / launch_s, "rows_per_launch": rows, "parts": rates}


# ------------------------------------------------------------ multi-rank

def max_over_ranks(x, world, device=None):
    """Largest x over all ranks (the slowest rank sets the job's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, batch, steps, t_max):
    """Queries per second of the whole job: every rank answers `batch`
    queries per step (weak scaling), all ranks finish within t_max."""
    return world * batch * steps / t_max


def rank_queries(n_u, batch, steps, rank):
    """Each rank's own query stream, [steps][batch] (replicas share no work)."""
    return synth.draw_queries(n_u, batch * steps, seed=11 + 1000 * rank).reshape(steps, batch)


# ------------------------------------------------------------------ ours

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2512_11606_gb300 import ahpp

    spec = graph_spec(args.graph, args.scale, args.scale_edges_only)
    g = synth.make_graph(**spec)

    cpu = None
    exact_pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = args.cpu_queries or min(16, host_cores())
        cpu = cpu_oracle_sample(g, args.eps, n)
        if not args.no_exact:
            # runs on the host cores while the GPU legs run (a few cores stay
            # free for the launching thread, the serving loop and the sampler)
            exact_pool = start_exact_refs(g, spec, cpu, args.cost_queries,
                                          max(1, host_cores() - 4))

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    G = ahpp.Graph.from_arrays(g, device=local_rank)
    tune = None
    if not args.no_autotune:
        # launch shapes tuned on a sample of the workload's queries (device-timed)
        t0 = time.perf_counter()
        G.autotune(synth.draw_queries(g.n_u, 32, seed=13 + rank), args.eps)
        tune = time.perf_counter() - t0
    info = G.info
    stream = torch.cuda.Stream(device=dev)
    B, K, W = args.batch, args.steps, args.warmup
    qs_all = rank_queries(g.n_u, B, W + K, rank)
    q_t = [torch.from_numpy(qs_all[i].astype(np.int32)).to(dev) for i in range(W + K)]
    eps_t = torch.full((B,), args.eps, dtype=torch.float64, device=dev)
    k_t = torch.full((B,), args.k, dtype=torch.int32, device=dev)
    nodes_t = torch.empty((B, args.k), dtype=torch.int32, device=dev)
    scores_t = torch.empty((B, args.k), dtype=torch.float32, device=dev)
    n_t = torch.empty((B,), dtype=torch.int32, device=dev)
    stats_t = torch.empty((B, ahpp.STATS_BYTES), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def step(i):
        G.query_batch_device(q_t[i], eps_t, k_t, args.k, nodes_t, scores_t, n_t, stats_t, stream)

    for i in range(W):
        step(i)
    stream.synchronize()

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(gpu_index(local_rank))
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    all_stats = []
    t0 = time.perf_counter()
    for j in range(K):
        with torch.cuda.stream(stream):
            ev[j][0].record(stream)
        step(W + j)
        with torch.cuda.stream(stream):
            ev[j][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(launch_ms) / 1e3
    stats = decode_stats(ahpp, stats_t)
    rounds = stats["rounds"].astype(np.int64)
    tile = int(info["batch_tile"])
    tile_rounds = int(sum(rounds[i:i + tile].max() for i in range(0, B, tile)))

    t_max = max_over_ranks(dev_s, world, dev)
    value = whole_job_value(world, B, K, t_max)

    # e2e through the host API: each step's query ids come from pinned host
    # memory, the library copies them in and the results out inside the call
    e2e = None
    if not args.no_e2e:
        pinned = torch.from_numpy(qs_all[W:].astype(np.int32)).pin_memory()
        host_q = [pinned[j].numpy().view(np.uint32) for j in range(K)]
        G.query_batch(host_q[0][:64], args.eps, args.k)       # warm the host path
        torch.cuda.synchronize()
        te = time.perf_counter()
        for j in range(K):
            G.query_batch(host_q[j], args.eps, args.k)
        te = max_over_ranks(time.perf_counter() - te, world, dev)
        e2e = {"value": whole_job_value(world, B, K, te), "unit": "queries/s",
               "h2d_bytes_per_step": B * (4 + 8 + 4),
               "d2h_bytes_per_step": B * (args.k * 8 + 4 + ahpp.STATS_BYTES)}

    # plain one-query-at-a-time GPU push on the same graph
    plain = None
    if rank == 0 and args.plain_queries > 0:
        pq = synth.draw_queries(g.n_u, args.plain_queries + 1, seed=77)
        pn = torch.empty(args.k, dtype=torch.int32, device=dev)
        ps = torch.empty(args.k, dtype=torch.float32, device=dev)
        pc = torch.empty(1, dtype=torch.int32, device=dev)
        pst = torch.empty((1, ahpp.STATS_BYTES), dtype=torch.uint8, device=dev)
        G.query_device(int(pq[0]), args.eps, args.k, pn, ps, pc, pst, stream)
        stream.synchronize()
        lat, p_rounds, p_dense = [], [], []
        for q in pq[1:]:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record(stream)
            G.query_device(int(q), args.eps, args.k, pn, ps, pc, pst, stream)
            with torch.cuda.stream(stream):
                b.record(stream)
            stream.synchronize()
            lat.append(a.elapsed_time(b))
            sd = decode_stats(ahpp, pst)[0]
            p_rounds.append(int(sd["rounds"]))
            p_dense.append(int(sd["dense_rounds"]))
        plain = {"qps": 1e3 / statistics.mean(lat), "p50_ms": statistics.median(lat),
                 "p99_ms": float(np.percentile(lat, 99)), "queries": len(lat),
                 "rounds_mean": statistics.mean(p_rounds), "dense_rounds_mean": statistics.mean(p_dense)}
        # roofline of the plain path's kernel: algorithmic bytes of its pull
        # rounds (push rounds are counted as zero: an underestimate) over the
        # measured time of the whole call (k_query1 + top-k)
        peak_p, peak_kind_p = measured_peak()
        alg_p = statistics.mean(p_dense) * q1_round_bytes(info)
        ach_p = alg_p / (statistics.mean(lat) / 1e3) / 1e9
        plain["roofline"] = {"bound": "hbm", "kernel": "k_query1", "achieved": ach_p, "peak": peak_p,
                             "unit": "GB/s", "frac": ach_p / peak_p,
                             "algorithmic_bytes_per_pull_round": q1_round_bytes(info),
                             "traffic": ncu_traffic("k_query1", args.graph, statistics.mean(p_dense)),
                             "traffic_note": ("ncu DRAM bytes per pull round of one query "
                                              "(profiles/k_query1_medium.md) x the mean pull rounds"),
                             "peak_source": peak_kind_p}

    # serving: open-loop Poisson arrivals on the same graph (continuous batching)
    served = None
    if rank == 0 and args.serve_seconds > 0:
        served = run_serving(ahpp, G, g, args, rate=args.serve_load * value / world)

    parity = None
    if cpu is not None:
        exact = exact32 = None
        if exact_pool is not None:
            pool, ar, jobs = exact_pool
            try:
                vals = ar.get(timeout=1800)
                exact = [v for (w, _, _), v in zip(jobs, vals) if w == "graph"]
                exact32 = [v for (w, _, _), v in zip(jobs, vals) if w == "fp32"]
            finally:
                pool.close()
                pool.join()
        parity = parity_vs_oracle(G, cpu, args.eps, args.k, exact, exact32)

    ablation = None
    if rank == 0 and args.ablation > 0:
        ablation = run_ablation(ahpp, g, args, info["lambda"], local_rank)

    scale_leg = None
    if rank == 0 and args.scale_leg > 0 and args.graph == "medium":
        scale_leg = run_scale_leg(ahpp, args, local_rank)

    # roofline of the dominant kernel (the batched persistent launch)
    peak, peak_kind = measured_peak()
    alg = tile_rounds * round_bytes(info, tile) + topk_bytes(info, B)   # one launch (last step)
    achieved = alg / (sum(launch_ms) / K / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": ncu_traffic("k_tiles", args.graph, tile_rounds),
            "traffic_note": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one 32-query tile "
                             "per tile-round (profiles/k_tiles_medium_tile32.md), scaled by the launch's "
                             "tile-rounds"),
            "peak_source": peak_kind,
            "kernel": "k_tiles (persistent: all rounds + top-k of one 1,024-query step)",
            "algorithmic_bytes_per_launch": alg,
            "tile_rounds_per_launch": tile_rounds}

    try:
        roof["l2_rows"] = row_roofline(ahpp, info, tile_rounds, sum(launch_ms) / K / 1e3, local_rank)
    except Exception as e:  # the HBM roofline above stands on its own
        roof["l2_rows"] = {"error": str(e)}
    # L2 -> SM bytes (ncu capture, scaled) against the measured rate of random
    # 128-byte row gathers from an L2-resident table of the t_V size
    l2_bytes = ncu_traffic("k_tiles", args.graph, tile_rounds, "l2_to_sm_bytes_per_unit")
    parts = roof["l2_rows"].get("parts") if isinstance(roof.get("l2_rows"), dict) else None
    if l2_bytes and parts:
        peak_l2 = parts[1]["peak_rows_per_s"] * 4 * int(info["batch_tile"]) / 1e9
        ach_l2 = l2_bytes / (sum(launch_ms) / K / 1e3) / 1e9
        roof["l2_sm"] = {"bound": "l2 -> sm bandwidth", "unit": "GB/s", "achieved": ach_l2, "peak": peak_l2,
                         "frac": ach_l2 / peak_l2,
                         "note": ("achieved = ncu l1tex__m_xbar2l1tex_read_bytes per tile-round x tile-rounds / "
                                  "launch time; peak = measured random 128-byte row gathers from an "
                                  "L2-resident table (byte-limited: 64-512 B rows reach the same GB/s)")}

    lat_ms = launch_ms
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "queries/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": 1e3 * t_max / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded Philox power-law graph; the paper's datasets are not available)",
        "config": workload_config(args, {
            "lambda": info["lambda"], "tile": info["batch_tile"], "batch_groups": info["batch_groups"],
            "batch_chunk": info["batch_chunk"],
            "single_dense_div": info["single_dense_div"], "single_attr_push": info["single_attr_push"],
            "single_vec_width": info["single_vec_width"],
            "autotune_s": tune and round(tune, 1),
            "autotune_ms_per_query": tune and {k: _r(v, 3) for k, v in G.autotune_report().items()},
            "launch_shape": "ahpp_autotune on 32 sample queries" if tune else "defaults"}),
        "gpu_launches": K,
        "clocks": clocks,
        "cpu_baseline": cpu and {k: cpu[k] for k in ("value", "unit", "cores", "cpu_model", "kind", "sample")},
        "e2e": e2e,
        "roofline": roof,
        "plain": plain,
        "served": served,
        "parity": parity,
        "ablation": ablation,
        "scale_leg": scale_leg,
        "p50_ms": statistics.median(lat_ms),
        "p99_ms": float(np.percentile(lat_ms, 99)),
        "latency_note": "batched: a query completes with its 1,024-query step",
        "rounds_mean": float(rounds.mean()),
        "rounds_max": int(rounds.max()),
        "not_converged": int((stats["status"] != 0).sum()),
        "mass_err_max": float(stats["mass_err"].max()),
        "wall_s": wall,
    }
    # the headline numbers, short and last on the line
    sat = (served or {}).get("saturated") or {}
    ol = (served or {}).get("open_loop") or {}
    ex = (parity or {}).get("exact") or {}
    pq = plain["qps"] if plain else None
    out.update({
        "batched_qps": _opt(value / world, 4),
        "plain_qps": _opt(pq, 4),
        "speedup_vs_plain": _opt(pq and value / world / pq, 3),
        "served_qps": _opt(served and served["qps"], 4),
        "served_p50_ms": _opt(sat.get("p50_ms"), 4),
        "served_p99_ms": _opt(sat.get("p99_ms"), 4),
        "served_speedup_vs_plain": _opt(pq and served and served["qps"] / pq, 3),
        "served_open_loop_qps": _opt(ol.get("qps"), 4),
        "served_open_loop_p50_ms": _opt(ol.get("p50_ms"), 4),
        "served_open_loop_p99_ms": _opt(ol.get("p99_ms"), 4),
        "hbm_frac_k_tiles": _opt(roof["frac"], 3),
        "hbm_frac_k_query1": _opt(plain and plain["roofline"]["frac"], 3),
        "parity_max_abs_err_vs_oracle": _opt(parity and parity["max_abs_err_vs_oracle"], 3),
        "parity_max_err_vs_exact": _opt(ex.get("max_err_vs_exact"), 3),
        "parity_min_err_vs_exact": _opt(ex.get("min_err_vs_exact"), 3),
        "topk_overlap_vs_exact": ex.get("topk_overlap_vs_exact_min"),
        "bf16_precision_cost_max": _opt(((parity or {}).get("bf16_precision_cost") or {}).get("max_abs"), 3),
        "large_quarter_batched_qps": _opt(scale_leg and scale_leg["batched_qps"], 4),
        "large_quarter_vs_plain": _opt(scale_leg and scale_leg["batched_vs_plain"], 3),
    })
    G.close()
    return out


def topk_overlap(nodes, ref, k, eps):
    """Overlap of a returned top-k with the top-k of the reference vector;
    nodes whose reference score lies within 2 eps of the k-th score count as
    interchangeable (ties of the approximation)."""
    kk = min(k, ref.shape[0])
    order = np.lexsort((np.arange(ref.shape[0]), -ref))
    kth = ref[order[kk - 1]]
    ok = set(np.nonzero(ref >= kth - 2 * eps)[0].tolist())
    return len(set(np.asarray(nodes).tolist()) & ok) / kk


def _r(x, d=3):
    """x rounded to d significant digits (keeps the bench line short)."""
    return float(f"{x:.{d}g}")


def _opt(x, d=3):
    """_r(x, d), or None when there is no value."""
    return None if x is None or x is False else _r(float(x), d)


def parity_vs_oracle(G, cpu, eps, k, exact=None, exact32=None):
    """The oracle's sample queries through the batched GPU path.

    vs the oracle push: per query the largest |gpu - oracle| over all of U
    and the top-k overlap.  vs exact AHPP (the oracle's Algorithm 1 run until
    (1 - alpha)^T <= 1e-10): Theorem 2 asks 0 <= pi - pi_hat <= eps, so the
    largest and smallest pi - pi_hat per query, and the top-k overlap with
    the exact top-k (the precision measure of Fig. 7).  bf16 precision cost:
    for the queries in exact32, the largest |pi_exact(bf16 weights) -
    pi_exact(FP32 weights)| and the top-k overlap between the two exact
    vectors: how far storing the attribute weights as bfloat16 moves the
    answer from the one the FP32 input defines."""
    qs = cpu["queries"]
    dense, _, _ = G.query_batch_dense(qs, eps)
    res = G.query_batch(qs, eps, k)
    errs, overlaps, hi, lo, ov_ex = [], [], [], [], []
    for i, ref in enumerate(cpu["pi"]):
        gpu = dense[i].astype(np.float64)
        errs.append(float(np.abs(gpu - ref).max()))
        overlaps.append(topk_overlap(res[i].nodes, ref, k, eps))
        if exact is not None:
            d = exact[i] - gpu
            hi.append(float(d.max()))
            lo.append(float(d.min()))
            ov_ex.append(topk_overlap(res[i].nodes, exact[i], k, eps))
    out = {"queries": len(qs), "eps": eps, "k": k, "bound_abs": 1e-6,
           "max_abs_err_vs_oracle": max(errs), "per_query_max_abs_err": [_r(x) for x in errs],
           "topk_overlap_min": min(overlaps),
           "note": "batched GPU results of the CPU-baseline sample vs the FP64 oracle push"}
    if exact is not None:
        out["exact"] = {
            "reference": f"oracle Algorithm 1, T = {exact_T()} ((1 - alpha)^T <= {EXACT_TAIL:g}), FP64",
            "max_err_vs_exact": max(hi), "min_err_vs_exact": min(lo),
            "per_query_max_err": [_r(x) for x in hi], "per_query_min_err": [_r(x) for x in lo],
            "topk_overlap_vs_exact_min": min(ov_ex),
            "bound": f"0 <= pi - pi_hat <= eps = {eps:g} (Theorem 2), FP32 rounding below"}
    if exact32:
        cost, ov = [], []
        for i, e32 in enumerate(exact32):
            cost.append(float(np.abs(exact[i] - e32).max()))
            order = np.lexsort((np.arange(e32.shape[0]), -e32))
            ov.append(topk_overlap(order[:k], exact[i], k, eps))
        out["bf16_precision_cost"] = {
            "queries": len(cost), "max_abs": max(cost), "per_query_max_abs": [_r(x) for x in cost],
            "topk_overlap_min": min(ov),
            "note": ("exact AHPP with the attribute weights rounded to bfloat16 (what the library "
                     "stores) vs with the FP32 weights of the same graph, both by the FP64 oracle")}
    return out


def run_ablation(ahpp, g, args, lam, device):
    """Single-query ablation on the same graph (Exp-2's question): ASRP with
    the switch budget as read (rule 0) and as printed (rule 1); APP(E), the
    stricter threshold without the switch (ASRP's rule 2); APP(S), APP's
    thresholds with the switch; and APP; per variant the mean rounds, switch
    round and the plain-path throughput over args.ablation queries."""
    import torch
    variants = [("ASRP, switch budget as read (default)", dict(algo=ahpp.AHPP_ASRP, switch_rule=0)),
                ("ASRP, switch budget as printed", dict(algo=ahpp.AHPP_ASRP, switch_rule=1)),
                ("APP(E): ASRP's eps / lambda threshold, never switch", dict(algo=ahpp.AHPP_ASRP, switch_rule=2)),
                ("APP(S): APP's thresholds with the synchronous switch", dict(algo=ahpp.AHPP_APP_S)),
                ("APP", dict(algo=ahpp.AHPP_APP))]
    qs = synth.draw_queries(g.n_u, args.ablation + 1, seed=303)
    dev = torch.device("cuda", device)
    out = []
    for name, cfg in variants:
        G = ahpp.Graph.from_arrays(g, lam=lam, device=device, **cfg)
        try:
            G.query(int(qs[0]), args.eps, 1)                   # warm-up
            rounds, sw, ms = [], [], []
            for q in qs[1:]:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                r = G.query(int(q), args.eps, args.k)
                b.record()
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
                rounds.append(r.stats["rounds"])
                sw.append(r.stats["switch_round"])
            out.append({"variant": name, "queries": len(ms), "qps": 1e3 / statistics.mean(ms),
                        "p50_ms": statistics.median(ms), "rounds_mean": statistics.mean(rounds),
                        "switch_round_mean": statistics.mean(sw)})
        finally:
            G.close()
    return out


def run_scale_leg(ahpp, args, device):
    """The large recipe (Zipf(2.0), 30 attributes per node) scaled by
    args.scale_leg: batched (128 queries, one step after one warm-up step)
    and plain (two queries after one warm-up) queries/s at the bench's eps,
    top-1,000 as in the large workload; the smallest graph of the
    scalability sweep (Exp-3's shape on synthetic graphs)."""
    import torch
    spec = synth.scaled(synth.LARGE, args.scale_leg)
    t0 = time.perf_counter()
    gl = synth.make_graph(**spec)
    gen_s = time.perf_counter() - t0
    G = ahpp.Graph.from_arrays(gl, device=device)
    try:
        qs = synth.draw_queries(gl.n_u, 128 * 2 + 3, seed=515)
        G.query_batch(qs[:128], args.eps, 1000)                 # warm-up step
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        res = G.query_batch(qs[128:256], args.eps, 1000)
        b.record()
        torch.cuda.synchronize()
        batched = 128 / (a.elapsed_time(b) / 1e3)
        G.query(int(qs[256]), args.eps, 1000)
        lat = []
        for q in qs[257:259]:
            a.record()
            G.query(int(q), args.eps, 1000)
            b.record()
            torch.cuda.synchronize()
            lat.append(a.elapsed_time(b))
        plain = 1e3 / statistics.mean(lat)
        return {"scale": args.scale_leg, "n_u": gl.n_u, "n_v": gl.n_v, "n_e": gl.n_e, "n_ea": gl.n_ea,
                "lambda": G.lam, "rounds_mean": float(np.mean([r.stats["rounds"] for r in res])),
                "batched_qps": batched, "plain_qps": plain, "batched_vs_plain": batched / plain,
                "generate_s": gen_s,
                "note": "large recipe scaled (|U|, |V|, |E|, |A|); 128-query batch and 2 plain queries, top-1,000"}
    finally:
        G.close()


def closed_loop(srv, qs, eps, ks, inflight):
    """Keep `inflight` requests submitted: take results in submit order and
    submit the next request as each result is taken.  Returns the completion
    times (s from the first submit), latencies (ms) and rounds per request."""
    n = len(qs)
    pending = [(srv.submit(int(qs[i]), float(eps[i]), int(ks[i])), int(ks[i])) for i in range(min(inflight, n))]
    nxt = len(pending)
    done_t, lat, rounds = [], [], []
    t0 = time.perf_counter()
    while pending:
        t, kk = pending.pop(0)
        r = srv.wait(t, kk)
        done_t.append(time.perf_counter() - t0)
        lat.append(r.stats["served_ms"])
        rounds.append(r.stats["rounds"])
        if nxt < n:
            pending.append((srv.submit(int(qs[nxt]), float(eps[nxt]), int(ks[nxt])), int(ks[nxt])))
            nxt += 1
    return done_t, lat, rounds


def burst_end(done_t, i, gap_s):
    """The last index of the burst of completions that index i belongs to
    (results of one server step arrive together; a gap above gap_s starts
    the next burst)."""
    while i + 1 < len(done_t) and done_t[i + 1] - done_t[i] <= gap_s:
        i += 1
    return i


def steady_state(done_t, lat, inflight, gap_s=1e-3):
    """qps and latency over the window after the first wave and before the
    drain (None when the run is too short for one).  Both window edges are
    moved to the end of a burst, so the window spans whole server steps: an
    edge inside a burst would count up to a whole step's results against a
    fraction of its time."""
    n = len(done_t)
    lo, hi = inflight, n - inflight
    if hi - lo < 8:
        return None
    a, b = burst_end(done_t, lo - 1, gap_s), burst_end(done_t, hi - 1, gap_s)
    if b - a < 8:
        a, b = lo - 1, hi - 1
    return {
        "qps": (b - a) / (done_t[b] - done_t[a]),
        "p50_ms": statistics.median(lat[a + 1:b + 1]),
        "p99_ms": float(np.percentile(lat[a + 1:b + 1], 99)),
        "queries": n, "window_queries": b - a, "in_flight": inflight,
    }


def run_serving(ahpp, G, g, args, rate):
    """Continuous batching through the server API.

    saturated: closed loop with every slot busy and as many requests queued
    besides (lanes that all finish in one step are refilled at the next
    step), so the queue never runs dry; completed
    queries/s and submit-to-result latency over a steady-state window
    (ramp-up and drain excluded).  saturated_short_queue: the same with only
    a quarter of the slots queued (lower latency; lanes that finish together wait a
    step for requests the clients have not yet resubmitted).  saturated_mix:
    as saturated, with the serving workload's per-request eps and k.
    open_loop_light / open_loop: Poisson arrivals at 5 % of capacity and at
    `rate` queries/s; completed queries/s and latency percentiles.
    """
    out = {"slots": None, "rounds_per_step": args.serve_rounds}
    srv = ahpp.Server(G, max_slots=args.serve_slots, rounds_per_step=args.serve_rounds)
    try:
        slots = srv.info()["slots"]
        out["slots"] = slots
        warm = [srv.submit(int(x), args.eps, args.k) for x in synth.draw_queries(g.n_u, 8, seed=99)]
        for t in warm:
            srv.wait(t, args.k)

        n_sat = max(4 * slots, int(args.serve_seconds * rate / max(args.serve_load, 1e-3) / 2))
        full_q = 2 * slots        # every slot busy, as many queued: all slots may finish in one step
        short_q = slots + max(4, slots // 4)
        eps_u = np.full(n_sat, args.eps)
        k_u = np.full(n_sat, args.k)

        qs = synth.draw_queries(g.n_u, n_sat, seed=202)
        clk = ClockSampler(gpu_index(G.info["device"]))
        clk.start()
        done_t, lat, _ = closed_loop(srv, qs, eps_u, k_u, full_q)
        sat_clocks = clk.stop()
        sat = steady_state(done_t, lat, full_q)
        if sat:
            sat["clocks"] = sat_clocks
            sat["note"] = ("closed loop, requests in flight = 2 x slots (the queue never runs dry); "
                           "qps over the steady-state window; latency includes the queue wait")
            out["saturated"] = sat

        done_t, lat, _ = closed_loop(srv, qs, eps_u, k_u, short_q)
        short = steady_state(done_t, lat, short_q)
        if short:
            short["note"] = "closed loop, requests in flight = slots + a quarter of them queued"
            out["saturated_short_queue"] = short

        # the serving workload's request mix: eps log-uniform in [1e-7, 1e-4],
        # k in {10, 100, 1000} (per-request eps and k in one tile)
        rng = np.random.default_rng(404)
        qm = synth.draw_queries(g.n_u, n_sat, seed=405)
        em = np.exp(rng.uniform(np.log(1e-7), np.log(1e-4), n_sat))
        km = rng.choice([10, 100, 1000], n_sat)
        done_t, lat, rounds = closed_loop(srv, qm, em, km, full_q)
        mix = steady_state(done_t, lat, full_q)
        if mix:
            mix["rounds_mean"] = float(np.mean(rounds))
            mix["note"] = "closed loop as saturated; eps log-uniform in [1e-7, 1e-4], k in {10, 100, 1000}"
            out["saturated_mix"] = mix

        # light load: Poisson arrivals at 5 % of the batched capacity; the server
        # answers most requests on the single-query path
        rate_l = 0.05 * rate / max(args.serve_load, 1e-3)
        n_l = max(16, int(rate_l * min(6.0, args.serve_seconds)))
        t_arr, ql, _, _ = synth.draw_stream(n_l, rate_l, g.n_u, seed=103)
        tickets = []
        t0 = time.perf_counter()
        for i in range(n_l):
            delay = t0 + t_arr[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(int(ql[i]), args.eps, args.k))
        lat = [srv.wait(t, args.k).stats["served_ms"] for t in tickets]
        out["open_loop_light"] = {
            "rate_qps": rate_l, "queries": n_l, "p50_ms": statistics.median(lat),
            "p99_ms": float(np.percentile(lat, 99)),
            "note": "Poisson arrivals at 5 % of the batched capacity (single-query path at light load)",
        }

        # open loop (Poisson arrivals)
        n = max(32, int(rate * args.serve_seconds))
        t_arr, q, _, _ = synth.draw_stream(n, rate, g.n_u, seed=101)
        tickets = []
        t0 = time.perf_counter()
        for i in range(n):
            delay = t0 + t_arr[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(int(q[i]), args.eps, args.k))
        lat = []
        for t in tickets:
            lat.append(srv.wait(t, args.k).stats["served_ms"])
        span = time.perf_counter() - t0
        out["open_loop"] = {
            "rate_qps": rate, "queries": n, "qps": n / span, "p50_ms": statistics.median(lat),
            "p99_ms": float(np.percentile(lat, 99)),
            "note": "Poisson arrivals at rate_qps; qps = completed / (last result - first submit)",
        }
        out["steps"] = srv.info()["steps"]
    finally:
        srv.stop()
    sat = out.get("saturated")
    out["qps"] = sat["qps"] if sat else out["open_loop"]["qps"]
    out["p50_ms"] = sat["p50_ms"] if sat else out["open_loop"]["p50_ms"]
    out["p99_ms"] = sat["p99_ms"] if sat else out["open_loop"]["p99_ms"]
    return out


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle on the host cores.

    A whole ASRP query takes the oracle tens of seconds on one core, so a
    step is a bounded slice of a continuous run: every host core keeps one
    query in flight, and a step advances each by R rounds from its kept state
    (og_push_resume; a query that converges is followed by the next one).
    R is sized from a short probe step so a step takes about
    --ref-step-seconds.  Queries/s = the rounds run in the timed steps over
    the mean rounds of a whole query (from the queries that converged), per
    wall second; over a window of several query lifetimes the steps cover
    every stage of a query's trajectory."""
    if rank != 0:
        return None
    spec = graph_spec(args.graph, args.scale, args.scale_edges_only)
    g = synth.make_graph(**spec)
    n = args.cpu_queries or min(16, host_cores())
    import oracle
    global _OG
    _OG = oracle.OracleGraph.from_arrays(g)
    lam, _ = _OG.lambda_estimate(ALPHA, BETA)
    ctx = mp.get_context("fork")
    qs = synth.draw_queries(g.n_u, n * 4096, seed=11).reshape(n, -1)
    cores = []
    for c in range(n):
        parent, child = ctx.Pipe()
        pr = ctx.Process(target=_ref_core, args=(child, qs[c], args.eps, lam), daemon=True)
        pr.start()
        cores.append((pr, parent))

    def step(budget):
        t0 = time.perf_counter()
        for _, conn in cores:
            conn.send(budget)
        out = [conn.recv() for _, conn in cores]
        return time.perf_counter() - t0, sum(o[1] for o in out), [r for o in out for r in o[2]]

    try:
        probe_rounds = 4
        t_probe, _, finished = step(probe_rounds)                 # sizes R (untimed)
        R = int(max(1, round(probe_rounds * args.ref_step_seconds / max(t_probe, 1e-9))))
        for _ in range(1, args.warmup):
            finished += step(R)[2]
        times, rounds_run = [], 0
        for _ in range(max(args.steps, 1)):
            dt, ran, fin = step(R)
            times.append(dt)
            rounds_run += ran
            finished += fin
        while not finished:                                       # a whole query's rounds (untimed)
            finished += step(R)[2]
    finally:
        for pr, conn in cores:
            try:
                conn.send(None)
            except Exception:
                pass
            pr.join(timeout=30)
    r_whole = statistics.mean(finished)
    total = sum(times)
    value = rounds_run / r_whole / total
    sample = (f"{n} ASRP queries in flight, one per host core (FP64); a step advances each by {R} rounds "
              f"from its kept state, the next query starting as one converges; queries/s = rounds in the "
              f"timed steps / {r_whole:.1f} rounds per whole query (mean of {len(finished)} that converged) "
              f"per wall second; lambda {lam:.2f}")
    return {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": workload_config(args, {"reference": "FP64 CPU oracle (the paper ships no code)"}),
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": n, "cpu_model": host_cpu_model(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
