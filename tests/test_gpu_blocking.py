"""Simpfer's norm-based blocking in place of the Cone-Tree (the paper's SA-Simpfer ablation,
Experiments, ablation study): blocks are runs of leaf_size users in descending norm order,
and the block and user bounds reduce to Cauchy-Schwarz (||q|| for a unit user).  Only the
pruning changes, so exact mode must still equal the FP64 oracle bit for bit.
"""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

VARIANTS = {
    "fp32": dict(precision=0),
    "bf16-simt": dict(precision=1, tc_user_pass=0),
    "bf16-tc": dict(precision=1, tc_user_pass=1),
}


def _truth(U, P, q, ks):
    c = oracle.count_above(U, P, q)
    return {int(k): np.flatnonzero(c < k).astype(np.int32) for k in ks}


def test_blocks_are_norm_runs(sah):
    W = workload.make("c2", m=3000, n=800)
    U = W.U.copy()
    U[17] = 0.0                      # a zero-norm user stays out of the blocks
    U[40] = U[41]                    # equal norms: the lower id first
    ix = sah.Index(U, W.P, k_max=50, leaf_size=64, blocking=sah.BLOCK_NORM)
    ids, starts, ct, cw = ix.blocks()
    norms = np.linalg.norm(U.astype(np.float64), axis=1)
    nz = np.flatnonzero(norms > 0)
    assert np.array_equal(np.sort(ids), nz)
    # descending norm (the library's FP32 norms may differ from these in the last bits)
    seq = norms[ids]
    assert np.all(seq[1:] <= seq[:-1] * (1 + 1e-6))
    pos = {int(u): i for i, u in enumerate(ids)}
    assert pos[40] < pos[41]                 # identical rows: the lower id first
    assert np.array_equal(starts, np.append(np.arange(0, len(nz), 64), len(nz)))
    assert np.all(ct == 0.0) and np.all(cw == -1.0)
    ix.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("p_prime", [10, 0, 1 << 30])
def test_norm_blocking_equals_oracle(sah, variant, p_prime):
    W = workload.make("c2", m=6000, n=2500)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=p_prime, seed=7, blocking=sah.BLOCK_NORM,
                   **VARIANTS[variant])
    ks = [1, 5, 10, 20, 50, 64]
    qidx = W.query_idx[:8]
    Q = np.repeat(W.P[qidx], len(ks), axis=0)
    K = np.tile(np.array(ks, np.int32), len(qidx))
    got = ix.rkmips_batch(Q, K)
    for a, qi in enumerate(qidx):
        want = _truth(W.U, W.P, W.P[qi], ks)
        for b, k in enumerate(ks):
            assert np.array_equal(got[a * len(ks) + b], want[k]), (qi, k, p_prime, variant)
    ix.close()


def test_rejects_unknown_blocking(sah):
    W = workload.make("c1", m=100, n=50)
    with pytest.raises(sah.SahError) as e:
        sah.Index(W.U, W.P, k_max=10, leaf_size=16, blocking=2)
    assert e.value.status == sah.SAH_ERR_ARG
