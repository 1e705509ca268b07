"""Python binding of the C ABI in include/ahpp.h (argument marshalling only).

Every computation runs in libahpp_gb300.so's CUDA kernels; this module only
converts numpy arrays / torch tensors to pointers and back.  Importing it
loads the library and raises if it is missing: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("AHPP_LIB") or os.path.join(HERE, "_build", "libahpp_gb300.so")

AHPP_OK, AHPP_EINVAL, AHPP_ENOMEM, AHPP_ECUDA = 0, -1, -2, -3
AHPP_ENOTCONVERGED, AHPP_EBUSY, AHPP_ETIMEOUT, AHPP_ESTATE = -4, -5, -6, -7
AHPP_ECANCELED = -8
AHPP_APP, AHPP_ASRP, AHPP_APP_S = 1, 2, 3
AHPP_MAX_K = 4096

_ERRNAMES = {AHPP_EINVAL: "EINVAL", AHPP_ENOMEM: "ENOMEM", AHPP_ECUDA: "ECUDA",
             AHPP_ENOTCONVERGED: "ENOTCONVERGED", AHPP_EBUSY: "EBUSY",
             AHPP_ETIMEOUT: "ETIMEOUT", AHPP_ESTATE: "ESTATE"}

_u32p = ctypes.POINTER(ctypes.c_uint32)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_u", ctypes.c_uint64), ("n_v", ctypes.c_uint64), ("n_a", ctypes.c_uint64),
                ("n_e", ctypes.c_uint64), ("e_u", _u32p), ("e_v", _u32p), ("e_w", _f32p),
                ("n_ea", ctypes.c_uint64), ("ea_u", _u32p), ("ea_a", _u32p), ("ea_w", _f32p)]


class Config(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("algo", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("lambda_T", ctypes.c_int),
                ("attr_bf16", ctypes.c_int), ("kahan", ctypes.c_int),
                ("switch_rule", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_uint64),
                ("device", ctypes.c_int), ("max_rounds", ctypes.c_uint32),
                ("batch_tile", ctypes.c_uint32), ("batch_groups", ctypes.c_uint32),
                ("batch_chunk", ctypes.c_uint32), ("single_vec_width", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("switch_round", ctypes.c_uint32),
                ("dense_rounds", ctypes.c_uint32), ("status", ctypes.c_uint32),
                ("pushes", ctypes.c_uint64), ("n_p", ctypes.c_uint64),
                ("resid_sum", ctypes.c_double), ("reserve_sum", ctypes.c_double),
                ("mass_err", ctypes.c_double), ("max_resid", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("eps_f", ctypes.c_double),
                ("served_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k.rstrip("_"): getattr(self, k) for k, _ in self._fields_}


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_u", ctypes.c_uint64), ("n_v", ctypes.c_uint64), ("n_a", ctypes.c_uint64),
                ("n_e", ctypes.c_uint64), ("n_ea", ctypes.c_uint64), ("lambda_", ctypes.c_double),
                ("lambda_T", ctypes.c_uint32), ("graph_bytes", ctypes.c_uint64),
                ("query_state_bytes", ctypes.c_uint64), ("tile_state_bytes", ctypes.c_uint64),
                ("device", ctypes.c_int), ("sm_count", ctypes.c_int),
                ("batch_tile", ctypes.c_uint32), ("batch_groups", ctypes.c_uint32),
                ("batch_chunk", ctypes.c_uint32),
                ("single_dense_div", ctypes.c_uint32), ("single_attr_push", ctypes.c_uint32),
                ("single_vec_width", ctypes.c_uint32), ("single_smem_bytes", ctypes.c_uint32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_uint32), ("queue_capacity", ctypes.c_uint32),
                ("tile", ctypes.c_uint32), ("rounds_per_step", ctypes.c_uint32),
                ("single_max", ctypes.c_int32)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("steps", ctypes.c_uint64),
                ("in_flight", ctypes.c_uint32), ("queued", ctypes.c_uint32),
                ("slots", ctypes.c_uint32)]


# Exported C symbols with (restype, argtypes): the full surface of include/ahpp.h.
SIGNATURES = {
    "ahpp_config_default": (None, [ctypes.POINTER(Config)]),
    "ahpp_last_error": (ctypes.c_char_p, []),
    "ahpp_load_graph": (ctypes.c_int, [ctypes.POINTER(GraphDesc), ctypes.POINTER(Config),
                                       ctypes.POINTER(_vp)]),
    "ahpp_save_graph": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "ahpp_load_graph_file": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(Config), ctypes.POINTER(_vp)]),
    "ahpp_free_graph": (None, [_vp]),
    "ahpp_get_graph_info": (ctypes.c_int, [_vp, ctypes.POINTER(GraphInfo)]),
    "ahpp_query": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint32,
                                  _u32p, _f32p, _u32p, ctypes.POINTER(Stats)]),
    "ahpp_query_dense": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_double, _f32p,
                                        ctypes.POINTER(Stats)]),
    "ahpp_query_batch": (ctypes.c_int, [_vp, ctypes.c_uint32, _u32p, _f64p, _u32p, _u32p, _f32p,
                                        _u32p, ctypes.POINTER(Stats)]),
    "ahpp_query_batch_dense": (ctypes.c_int, [_vp, ctypes.c_uint32, _u32p, _f64p, _f32p,
                                              ctypes.POINTER(Stats)]),
    "ahpp_query_batch_device": (ctypes.c_int, [_vp, ctypes.c_uint32, _vp, _vp, _vp,
                                               ctypes.c_uint32, _vp, _vp, _vp, _vp, _vp]),
    "ahpp_query_device": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint32,
                                         _vp, _vp, _vp, _vp, _vp]),
    "ahpp_query_dense_noalloc": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_double, _vp, _vp]),
    "ahpp_autotune": (ctypes.c_int, [_vp, ctypes.c_uint32, _u32p, ctypes.c_double]),
    "ahpp_autotune_report": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_size_t)]),
    "ahpp_server_start": (ctypes.c_int, [_vp, ctypes.POINTER(ServerOpts), ctypes.POINTER(_vp)]),
    "ahpp_submit": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint32,
                                   _u64p]),
    "ahpp_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_int, _u32p, _f32p, _u32p,
                                 ctypes.POINTER(Stats)]),
    "ahpp_server_info_get": (ctypes.c_int, [_vp, ctypes.POINTER(ServerInfo)]),
    "ahpp_server_stop": (ctypes.c_int, [_vp]),
    "ahpp_cancel": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "ahpp_power_iteration": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, _f32p,
                                            ctypes.POINTER(Stats)]),
    "ahpp_row_access_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_double)]),
    "ahpp_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                  ctypes.POINTER(ctypes.c_int)]),
    "ahpp_selftest_arm_wait_timeout": (ctypes.c_int, [_vp]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libahpp_gb300.so and declare every exported function."""
    if not os.path.exists(path):
        raise ImportError(f"libahpp_gb300.so not built ({path}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class AhppError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def _check(rc: int, allow=()) -> int:
    if rc != AHPP_OK and rc not in allow:
        raise AhppError(rc, lib().ahpp_last_error().decode())
    return rc


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def default_config(**kw) -> Config:
    c = Config()
    lib().ahpp_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, "lambda_" if k == "lam" else k, v)
    return c


@dataclass
class QueryResult:
    nodes: np.ndarray
    scores: np.ndarray
    stats: dict
    rc: int


class Graph:
    """A graph loaded on the GPU (owns all its device memory)."""

    def __init__(self, n_u, n_v, n_a, e_u, e_v, e_w, ea_u, ea_a, ea_w, config: Config | None = None,
                 **cfg):
        self._keep = [np.ascontiguousarray(e_u, np.uint32), np.ascontiguousarray(e_v, np.uint32),
                      None if e_w is None else np.ascontiguousarray(e_w, np.float32),
                      np.ascontiguousarray(ea_u, np.uint32), np.ascontiguousarray(ea_a, np.uint32),
                      None if ea_w is None else np.ascontiguousarray(ea_w, np.float32)]
        eu, ev, ew, au, aa, aw = self._keep
        d = GraphDesc(n_u, n_v, n_a, eu.shape[0], _p(eu, _u32p), _p(ev, _u32p),
                      None if ew is None else _p(ew, _f32p), au.shape[0], _p(au, _u32p),
                      _p(aa, _u32p), None if aw is None else _p(aw, _f32p))
        self.config = config if config is not None else default_config(**cfg)
        h = _vp()
        _check(lib().ahpp_load_graph(ctypes.byref(d), ctypes.byref(self.config), ctypes.byref(h)))
        self._h = h
        self._keep = None
        self.info = self.get_info()

    @classmethod
    def load_file(cls, path: str, **cfg) -> "Graph":
        """A graph saved by save(); alpha, beta and attr_bf16 must match it."""
        self = cls.__new__(cls)
        self.config = default_config(**cfg)
        h = _vp()
        _check(lib().ahpp_load_graph_file(os.fsencode(path), ctypes.byref(self.config), ctypes.byref(h)))
        self._h = h
        self._keep = None
        self.info = self.get_info()
        return self

    def save(self, path: str) -> None:
        _check(lib().ahpp_save_graph(self._h, os.fsencode(path)))

    @classmethod
    def from_arrays(cls, g, **cfg) -> "Graph":
        return cls(g.n_u, g.n_v, g.n_a, g.e_u, g.e_v, g.e_w, g.ea_u, g.ea_a, g.ea_w, **cfg)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ahpp_free_graph(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_info(self) -> dict:
        i = GraphInfo()
        _check(lib().ahpp_get_graph_info(self._h, ctypes.byref(i)))
        return {k.rstrip("_"): getattr(i, k) for k, _ in i._fields_}

    @property
    def n_u(self) -> int:
        return int(self.info["n_u"])

    @property
    def lam(self) -> float:
        return float(self.info["lambda"])

    def query(self, q: int, eps: float, k: int) -> QueryResult:
        kk = min(k, self.n_u)
        nodes = np.zeros(max(kk, 1), np.uint32)
        scores = np.zeros(max(kk, 1), np.float32)
        n = ctypes.c_uint32(0)
        st = Stats()
        rc = _check(lib().ahpp_query(self._h, q, eps, k, _p(nodes, _u32p), _p(scores, _f32p),
                                     ctypes.byref(n), ctypes.byref(st)), (AHPP_ENOTCONVERGED,))
        return QueryResult(nodes[: n.value], scores[: n.value], st.as_dict(), rc)

    def query_dense(self, q: int, eps: float):
        out = np.zeros(self.n_u, np.float32)
        st = Stats()
        rc = _check(lib().ahpp_query_dense(self._h, q, eps, _p(out, _f32p), ctypes.byref(st)),
                    (AHPP_ENOTCONVERGED,))
        return out, st.as_dict(), rc

    def power_iteration(self, q: int, T: int):
        """Algorithm 1's iterate after T iterations from q (dense, caller ids)."""
        out = np.zeros(self.n_u, np.float32)
        st = Stats()
        rc = _check(lib().ahpp_power_iteration(self._h, q, T, _p(out, _f32p), ctypes.byref(st)))
        return out, st.as_dict(), rc

    def query_batch(self, q, eps, k):
        q = np.ascontiguousarray(q, np.uint32)
        n = q.shape[0]
        eps = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (n,)))
        k = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.uint32), (n,)))
        kk = np.minimum(k, self.n_u)
        tot = int(kk.sum())
        nodes = np.zeros(max(tot, 1), np.uint32)
        scores = np.zeros(max(tot, 1), np.float32)
        cnt = np.zeros(n, np.uint32)
        st = (Stats * max(n, 1))()
        rc = _check(lib().ahpp_query_batch(self._h, n, _p(q, _u32p), _p(eps, _f64p), _p(k, _u32p),
                                           _p(nodes, _u32p), _p(scores, _f32p), _p(cnt, _u32p), st),
                    (AHPP_ENOTCONVERGED,))
        off = np.concatenate([np.zeros(1, np.int64), np.cumsum(cnt, dtype=np.int64)])
        res = [QueryResult(nodes[off[i]:off[i + 1]], scores[off[i]:off[i + 1]], st[i].as_dict(), rc)
               for i in range(n)]
        return res

    def query_batch_dense(self, q, eps):
        q = np.ascontiguousarray(q, np.uint32)
        n = q.shape[0]
        eps = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (n,)))
        out = np.zeros((n, self.n_u), np.float32)
        st = (Stats * max(n, 1))()
        rc = _check(lib().ahpp_query_batch_dense(self._h, n, _p(q, _u32p), _p(eps, _f64p),
                                                 _p(out, _f32p), st), (AHPP_ENOTCONVERGED,))
        return out, [st[i].as_dict() for i in range(n)], rc

    # ---- device-resident variants (torch tensors on the graph's device)
    def query_batch_device(self, q_t, eps_t, k_t, kmax, nodes_t, scores_t, n_t, stats_t=None,
                           stream=None) -> int:
        return _check(lib().ahpp_query_batch_device(
            self._h, int(q_t.numel()), q_t.data_ptr(), eps_t.data_ptr(), k_t.data_ptr(), kmax,
            nodes_t.data_ptr(), scores_t.data_ptr(), n_t.data_ptr(),
            None if stats_t is None else stats_t.data_ptr(),
            None if stream is None else stream.cuda_stream), (AHPP_ENOTCONVERGED,))

    def query_device(self, q, eps, k, nodes_t, scores_t, n_t, stats_t=None, stream=None) -> int:
        return _check(lib().ahpp_query_device(
            self._h, q, eps, k, nodes_t.data_ptr(), scores_t.data_ptr(), n_t.data_ptr(),
            None if stats_t is None else stats_t.data_ptr(),
            None if stream is None else stream.cuda_stream), (AHPP_ENOTCONVERGED,))

    def query_dense_noalloc(self, q, eps, out_t, stream=None) -> int:
        """Dense reserves into the caller's device tensor out_t[n_u] with no
        device allocation (the query state lives in the library's static
        scratch array)."""
        return _check(lib().ahpp_query_dense_noalloc(
            self._h, q, eps, out_t.data_ptr(), None if stream is None else stream.cuda_stream),
            (AHPP_ENOTCONVERGED,))

    def arm_wait_timeout(self) -> None:
        """Self-test: the next persistent launch on this graph starts with a
        grid barrier that can never fill, so its call reports AHPP_ETIMEOUT
        after about a second (ahpp_selftest_arm_wait_timeout)."""
        _check(lib().ahpp_selftest_arm_wait_timeout(self._h))

    def autotune(self, q_sample, eps: float) -> dict:
        q = np.ascontiguousarray(q_sample, np.uint32)
        _check(lib().ahpp_autotune(self._h, q.shape[0], _p(q, _u32p), eps))
        self.info = self.get_info()
        return self.info

    def autotune_report(self) -> dict:
        """ms of device time per query of every candidate the last autotune timed."""
        n = ctypes.c_size_t(0)
        _check(lib().ahpp_autotune_report(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value + 1)
        _check(lib().ahpp_autotune_report(self._h, buf, n.value + 1, None))
        import json
        return json.loads(buf.value.decode() or "{}")


STATS_BYTES = ctypes.sizeof(Stats)


def selftest_wait_timeout(device: int = 0):
    """(blocks that reported a given-up device wait, context usable after)."""
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().ahpp_selftest_wait_timeout(device, ctypes.byref(a), ctypes.byref(b)))
    return a.value, bool(b.value)


def row_access_peak(table_bytes: int, op: str = "gather", device: int = 0) -> float:
    """Random 128-byte row gathers (op "gather") or float4 row reductions
    (op "reduce") per second on `device`, from / into a table of table_bytes."""
    out = ctypes.c_double(0.0)
    _check(lib().ahpp_row_access_peak(device, int(table_bytes), {"gather": 0, "reduce": 1}[op],
                                      ctypes.byref(out)))
    return out.value


class Server:
    """Continuous-batching server over a loaded graph."""

    def __init__(self, graph: Graph, max_slots: int = 0, queue_capacity: int = 0, tile: int = 0,
                 rounds_per_step: int = 0, single_max: int = 0):
        self.graph = graph
        o = ServerOpts(max_slots, queue_capacity, tile, rounds_per_step, single_max)
        h = _vp()
        _check(lib().ahpp_server_start(graph.handle, ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def submit(self, q: int, eps: float, k: int) -> int:
        t = ctypes.c_uint64(0)
        _check(lib().ahpp_submit(self._h, q, eps, k, ctypes.byref(t)))
        return t.value

    def try_submit(self, q: int, eps: float, k: int):
        t = ctypes.c_uint64(0)
        rc = lib().ahpp_submit(self._h, q, eps, k, ctypes.byref(t))
        if rc == AHPP_EBUSY:
            return None
        _check(rc)
        return t.value

    def wait(self, ticket: int, k: int, timeout_ms: int = -1):
        nodes = np.zeros(max(k, 1), np.uint32)
        scores = np.zeros(max(k, 1), np.float32)
        n = ctypes.c_uint32(0)
        st = Stats()
        rc = lib().ahpp_wait(self._h, ticket, timeout_ms, _p(nodes, _u32p), _p(scores, _f32p),
                             ctypes.byref(n), ctypes.byref(st))
        if rc == AHPP_ETIMEOUT:
            return None
        _check(rc, (AHPP_ENOTCONVERGED, AHPP_ECANCELED))
        return QueryResult(nodes[: n.value], scores[: n.value], st.as_dict(), rc)

    def cancel(self, ticket: int) -> int:
        """Drop a queued request or free its slot at the next step; its wait
        then returns rc AHPP_ECANCELED (unless it finished first)."""
        return _check(lib().ahpp_cancel(self._h, ticket))

    def info(self) -> dict:
        i = ServerInfo()
        _check(lib().ahpp_server_info_get(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in i._fields_}

    def stop(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ahpp_server_stop(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
