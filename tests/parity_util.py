"""Shared parity checks of the GPU tests (test infrastructure).

The bar (the same at every eps): every score within TOL = 1e-6 absolute of
the reference it is compared with (the FP64 oracle push, or the same query
through another GPU path), element by element.  A top-k list is checked
entry by entry against the reference's dense vector, for its order, and for
its overlap with the reference's top-k (>= 0.99), where nodes whose
reference score lies within 2 max(eps, TOL) of the k-th score are
interchangeable (the tie rule of the top-k comparison: scores that close are
not ordered by an eps-approximation).
"""
import numpy as np

TOL = 1e-6
MIN_OVERLAP = 0.99


def check_topk(nodes, scores, ref, k, eps, tol=TOL, min_overlap=MIN_OVERLAP):
    """A returned top-k (nodes, scores) against the dense reference vector
    ref; returns the overlap."""
    nodes = np.asarray(nodes, dtype=np.int64)
    scores = np.asarray(scores, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    k = min(int(k), ref.shape[0])
    assert nodes.shape[0] == k, (nodes.shape[0], k)
    assert len(set(nodes.tolist())) == k                       # distinct nodes
    d = np.abs(scores - ref[nodes]).max() if k else 0.0
    assert d <= tol, d
    # score descending, then node id ascending
    assert np.all(np.lexsort((nodes, -scores)) == np.arange(k))
    w = 2.0 * max(eps, tol)
    order = np.lexsort((np.arange(ref.shape[0]), -ref))
    kth = ref[order[k - 1]]
    sure = set(order[:k][ref[order[:k]] > kth + w].tolist())   # in every valid top-k
    ok = set(np.nonzero(ref >= kth - w)[0].tolist())
    got = set(nodes.tolist())
    missing = sure - got
    assert not missing, sorted(missing)[:10]
    overlap = len(got & ok) / k
    assert overlap >= min_overlap, overlap
    return overlap


def check_dense(gpu, ref, tol=TOL):
    """Element-wise |gpu - ref| <= tol over the whole vector; returns the max."""
    d = float(np.abs(np.asarray(gpu, np.float64) - np.asarray(ref, np.float64)).max())
    assert d <= tol, d
    return d
