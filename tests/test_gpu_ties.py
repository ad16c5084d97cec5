"""Exact thresholds with queries that are items, some of them duplicated: a user whose k-th
item is the query (or a copy of it) scores exactly its threshold, and the pair is settled by
the double-precision re-score, whose sequential sum reproduces the threshold bit for bit.
Every answer is checked against the FP64 oracle (the count rule is strict, so copies of q
never count against it)."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("leaf", [16, 64])
def test_item_queries_with_duplicates(sah, leaf):
    W = workload.make("c1", m=1500, n=900)
    P = W.P.copy()
    P[10:20] = P[100:110]        # ten items present twice
    P[30] = P[31] = P[32]        # one present three times
    ix = sah.Index(W.U, P, k_max=20, leaf_size=leaf, p_prime=1 << 30, precision=1, tc_user_pass=1)
    rows = [10, 11, 100, 101, 30, 31, 32, 5, 300, 899]
    ks = [1, 2, 5, 13, 20]
    Q = np.ascontiguousarray(np.repeat(P[rows], len(ks), axis=0))
    K = np.tile(np.array(ks, np.int32), len(rows))
    got = ix.rkmips_batch(Q, K)
    for i in range(len(K)):
        want = np.flatnonzero(oracle.count_above(W.U, P, Q[i]) < K[i]).astype(np.int32)
        assert np.array_equal(got[i], want), (i, int(K[i]))
    # the same batch again (replayed graph) and through device buffers
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    total = sum(len(g) for g in got)
    out = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    offs = torch.empty(len(K) + 1, dtype=torch.int64, device=dev)
    for _ in range(2):
        ix.rkmips_batch_device(torch.from_numpy(Q).to(dev), torch.from_numpy(K).to(dev), out, offs)
        o = offs.cpu().numpy()
        ids = out.cpu().numpy()
        for i in range(len(K)):
            assert np.array_equal(ids[o[i]:o[i + 1]], got[i]), i
