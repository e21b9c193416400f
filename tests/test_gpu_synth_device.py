"""The device-side rating generator (used for the 10^8-cell and batched
workloads): exact cell count, consistent user/item CSRs, the rating recipe,
the 90/10 split, and determinism for a seed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_18024_gb300 import synth

pytestmark = pytest.mark.gpu


def host(t):
    return t.cpu().numpy()


def cells(indptr, indices, values):
    rows = np.repeat(np.arange(len(indptr) - 1), np.diff(indptr))
    return rows, indices.astype(np.int64), values


def test_device_generator_properties():
    n_u, n_m, nnz = 3000, 1200, 90_000
    p = synth.zipf_ratings_device(n_u, n_m, 8, nnz, 0.9, 0.5, seed=5)
    ip, ix, v = (host(t) for t in p.rows)
    jp, jx, w = (host(t) for t in p.cols)
    n_test = int(round(nnz * 0.1))
    assert ip[0] == 0 and ip[-1] == nnz - n_test and np.all(np.diff(ip) >= 0) and len(ip) == n_u + 1
    assert jp[0] == 0 and jp[-1] == nnz - n_test and len(jp) == n_m + 1
    assert len(host(p.test_u)) == n_test
    # Sorted, distinct column ids inside every row of both sides.
    for ptr, idx, n_other in ((ip, ix, n_m), (jp, jx, n_u)):
        assert idx.min() >= 0 and idx.max() < n_other
        d = np.diff(idx.astype(np.int64))
        starts = np.zeros(len(idx), bool)
        starts[ptr[:-1][np.diff(ptr) > 0]] = True
        assert np.all((d > 0) | starts[1:])
    # The item side is the transpose of the user side (same cells, same ratings).
    ru, cu, vu = cells(ip, ix, v)
    ci, ri, vi = cells(jp, jx, w)
    a = np.lexsort((cu, ru))
    b = np.lexsort((ci, ri))
    assert np.array_equal(ru[a], ri[b]) and np.array_equal(cu[a], ci[b]) and np.array_equal(vu[a], vi[b])
    # Test cells are disjoint from training cells; ratings are integers 1..5.
    train = set((ru * n_m + cu).tolist())
    test = host(p.test_u).astype(np.int64) * n_m + host(p.test_m).astype(np.int64)
    assert len(set(test.tolist())) == n_test and not (set(test.tolist()) & train)
    allr = np.concatenate([v, host(p.test_r)])
    assert np.all(allr == np.round(allr)) and allr.min() >= 1 and allr.max() <= 5
    # Deterministic for a seed, different for another.
    q = synth.zipf_ratings_device(n_u, n_m, 8, nnz, 0.9, 0.5, seed=5)
    assert all(torch.equal(x, y) for x, y in zip(p.rows, q.rows))
    r = synth.zipf_ratings_device(n_u, n_m, 8, nnz, 0.9, 0.5, seed=6)
    assert not torch.equal(p.rows[1], r.rows[1])


def test_device_generator_refuses_impossible_counts():
    with pytest.raises(ValueError):
        synth.zipf_ratings_device(10, 10, 4, 101, 0.9, 0.5, seed=1)
