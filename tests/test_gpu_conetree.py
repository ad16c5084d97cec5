"""The GPU Cone-Tree (Alg. 3, built level by level) against the oracle's recursive Alg. 3.

Both sides draw the random point of every node from the same SplitMix64 definition, keep
list order in the split and break argmin ties by position, so on inputs without near
ties the leaves agree exactly; leaf cones agree to FP32 accuracy."""
import numpy as np
import pytest

from oracle import sah as ref
import workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,N0,d", [(0, 20, 8), (3, 7, 5), (11, 64, 16), (5, 1, 4)])
def test_leaves_match_oracle(sah, seed, N0, d):
    W = workload.make("c1", m=1500, n=50, d=d, seed=seed)
    ix = sah.Index(W.U, W.P, k_max=10, leaf_size=N0, seed=seed)
    ids, starts, ct, cw = ix.blocks()
    U = W.U.astype(np.float64)
    Uhat = U / np.linalg.norm(U, axis=1, keepdims=True)
    leaves = ref.cone_tree(Uhat, np.arange(W.m), N0, seed)
    assert len(leaves) == len(starts) - 1
    for b, leaf in enumerate(leaves):
        got = ids[starts[b]:starts[b + 1]]
        assert np.array_equal(got, leaf.members), b
        assert abs(np.cos(leaf.omega) - cw[b]) < 2e-5
        assert np.allclose(np.cos(leaf.theta), ct[starts[b]:starts[b + 1]], atol=2e-5)


def test_tree_invariants_full_size_leaf_256(sah):
    W = workload.make("c2", m=100000, n=100)
    ix = sah.Index(W.U, W.P, k_max=10, leaf_size=256)
    ids, starts, ct, cw = ix.blocks()
    assert np.array_equal(np.sort(ids), np.arange(W.m))                 # disjoint cover
    sizes = np.diff(starts)
    assert sizes.min() >= 1 and sizes.max() <= 256
    for b in range(len(sizes)):
        assert np.all(ct[starts[b]:starts[b + 1]] >= cw[b] - 1e-6)      # theta_u <= omega
