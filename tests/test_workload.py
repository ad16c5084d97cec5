"""The seeded input generators that the oracle and the CUDA path share: the same seed gives
the same arrays, and the bench's workload keeps its shapes and request mix."""
import numpy as np

import workload


def test_same_seed_same_arrays_other_seed_differs():
    a = workload.make("c1", m=300, n=200)
    b = workload.make("c1", m=300, n=200)
    c = workload.make("c1", m=300, n=200, seed=1)
    assert np.array_equal(a.P, b.P) and np.array_equal(a.U, b.U)
    assert np.array_equal(a.query_idx, b.query_idx) and np.array_equal(a.ks, b.ks)
    assert not np.array_equal(a.P, c.P)


def test_bench_workload_shapes_and_requests():
    W = workload.make("c2", m=4000)   # C2's recipe at a smaller user count
    assert (W.n, W.d) == (17770, 50) and W.m == 4000
    assert W.P.dtype == np.float32 and W.U.dtype == np.float32
    assert W.P.flags.c_contiguous and W.U.flags.c_contiguous
    assert np.isfinite(W.P).all() and np.isfinite(W.U).all()
    assert len(W.query_idx) == 100 and len(set(W.query_idx.tolist())) == 100
    assert W.query_idx.min() >= 0 and W.query_idx.max() < W.n
    Q, K, rows = W.requests()
    assert Q.shape == (500, 50) and K.dtype == np.int32
    assert sorted(set(K.tolist())) == [1, 5, 10, 20, 50]
    # each item is asked at every k, its rows adjacent
    assert np.array_equal(Q[rows == 0], np.repeat(W.P[W.query_idx[:1]], 5, axis=0))
    # log-normal norms, with 5 % of the items at three times theirs: a heavy upper tail
    pn = np.linalg.norm(W.P.astype(np.float64), axis=1)
    assert np.quantile(pn, 0.99) > 2.0 * np.median(pn)
