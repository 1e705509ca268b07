"""The allocation-free single-query entry point (ahpp_query_dense_noalloc).

It serves callers that cannot allocate device memory at query time (a
framework owning the whole memory pool, or a thread that must not take the
synchronisation cudaMalloc / cudaFree may cause).  Its result must match the
allocating entry point (ahpp_query_dense) within the tolerance of the other
GPU tests, call after call, since every call reuses the same static scratch.
This file is collected last so that a failure here does not hide others.
"""
import numpy as np
import pytest

from paper_2512_11606_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-6


@pytest.fixture(scope="module")
def ahpp():
    from paper_2512_11606_gb300 import build
    build.build()
    from paper_2512_11606_gb300 import ahpp as mod
    return mod


def test_noalloc_matches_allocating_path_twice(ahpp):
    torch = pytest.importorskip("torch")
    g = synth.make_graph(**synth.TINY)
    G = ahpp.Graph.from_arrays(g, attr_bf16=0)
    try:
        out = torch.empty(g.n_u, dtype=torch.float32, device="cuda")
        for q in [int(x) for x in synth.draw_queries(g.n_u, 2, seed=21)]:
            out.fill_(-1.0)
            rc = G.query_dense_noalloc(q, 1e-6, out)
            assert rc == ahpp.AHPP_OK
            got = out.cpu().numpy()
            ref, st, rc2 = G.query_dense(q, 1e-6)
            assert rc2 == ahpp.AHPP_OK
            assert np.abs(got.astype(np.float64) - ref).max() <= TOL
            assert got.min() >= 0.0 and got[q] >= 0.15 - TOL
    finally:
        G.close()


def test_noalloc_rejects_graph_beyond_scratch(ahpp):
    torch = pytest.importorskip("torch")
    n = 3_000_000                       # 4 B x (4 |U| + ...) of state exceeds 32 MiB
    u = np.arange(n, dtype=np.uint32)
    z = np.zeros(n, dtype=np.uint32)
    one = np.ones(n, dtype=np.float32)
    G = ahpp.Graph(n, 1, 1, u, z, one, u, z, one)
    try:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        with pytest.raises(ahpp.AhppError) as e:
            G.query_dense_noalloc(0, 1e-3, out)
        assert e.value.code == ahpp.AHPP_EINVAL and "static scratch" in str(e.value)
    finally:
        G.close()


def test_noalloc_on_a_caller_stream_and_after_a_wait_timeout(ahpp):
    """A call on a stream the caller created gives the allocating path's
    result; a call whose first device wait gives up (self-test trap) reports
    AHPP_ETIMEOUT rather than the status an earlier call left in the shared
    scratch, and the next call is correct again."""
    torch = pytest.importorskip("torch")
    g = synth.make_graph(**synth.TINY)
    G = ahpp.Graph.from_arrays(g, attr_bf16=0)
    try:
        q = int(synth.draw_queries(g.n_u, 1, seed=22)[0])
        ref, _, rc = G.query_dense(q, 1e-6)
        assert rc == ahpp.AHPP_OK
        stream = torch.cuda.Stream()
        out = torch.empty(g.n_u, dtype=torch.float32, device="cuda")
        out.fill_(-1.0)
        stream.wait_stream(torch.cuda.current_stream())
        assert G.query_dense_noalloc(q, 1e-6, out, stream=stream) == ahpp.AHPP_OK
        got = out.cpu().numpy()
        assert np.abs(got.astype(np.float64) - ref).max() <= TOL
        G.arm_wait_timeout()
        with pytest.raises(ahpp.AhppError) as e:
            G.query_dense_noalloc(q, 1e-6, out, stream=stream)
        assert e.value.code == ahpp.AHPP_ETIMEOUT
        out.fill_(-1.0)
        stream.wait_stream(torch.cuda.current_stream())
        assert G.query_dense_noalloc(q, 1e-6, out, stream=stream) == ahpp.AHPP_OK
        assert np.abs(out.cpu().numpy().astype(np.float64) - ref).max() <= TOL
    finally:
        G.close()
