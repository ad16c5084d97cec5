"""The failure path of the bounded device-side waits, driven to expiry without a GPU fault.

Every wait inside a tensor-core kernel gives up after a bounded spin, raises the index's
device flag, drains its CTA's own TMA loads and MMAs and frees its tensor memory; the call
then returns SAH_ERR_DEVICE_TIMEOUT.  sah_index_inject_stall makes the MMA thread of one
pass stop after its first accumulator tile, so that its epilogue waits on a barrier that
nothing will complete: the wait runs out.  The next call on the same index must answer
exactly as the FP64 oracle does.
"""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def _oracle_sets(W, qrows, ks):
    out = {}
    for qi in qrows:
        c = oracle.count_above(W.U, W.P, W.P[qi])
        for k in ks:
            out[(int(qi), k)] = np.flatnonzero(c < k)
    return out


def _batch(W, qrows, ks):
    Q = np.repeat(W.P[qrows], len(ks), axis=0)
    K = np.tile(np.array(ks, np.int32), len(qrows))
    return Q, K


@pytest.mark.parametrize("site,p_prime", [(1, 1 << 30), (2, 0)])
def test_stalled_pass_times_out_and_index_recovers(sah, site, p_prime):
    # 60,000 users: about three 128-user tiles per CTA in the user pass; the paper's |P'|
    # (p_prime 0) leaves survivors whose kMIPS decision scans several item tiles
    W = workload.make("c2", m=60000, n=1500)
    qrows = W.query_idx[:3]
    ks = [10, 50]
    Q, K = _batch(W, qrows, ks)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=p_prime, precision=sah.BF16, tc_user_pass=1)
    want = _oracle_sets(W, qrows, ks)
    # a normal call first: the shapes repeat, so later calls would replay a CUDA graph
    # (the hooked call must not)
    for _ in range(2):
        got = ix.rkmips_batch(Q, K)
    ix.inject_stall(site)
    with pytest.raises(sah.SahError) as e:
        ix.rkmips_batch(Q, K)
    assert e.value.status == sah.SAH_ERR_DEVICE_TIMEOUT
    # the hook cleared itself; the index answers exactly, twice (direct, then replayed)
    for _ in range(2):
        got = ix.rkmips_batch(Q, K)
        for a, qi in enumerate(qrows):
            for b, k in enumerate(ks):
                assert np.array_equal(got[a * len(ks) + b], want[(int(qi), k)]), (site, qi, k)
    if site == 2:
        assert ix.stats()["survivors"] > 0      # the kMIPS decision did run
    ix.close()


def test_inject_stall_rejects_unknown_sites(sah):
    W = workload.make("c1", m=200, n=100)
    ix = sah.Index(W.U, W.P, k_max=10, leaf_size=32)
    for site in (-1, 3):
        with pytest.raises(sah.SahError) as e:
            ix.inject_stall(site)
        assert e.value.status == sah.SAH_ERR_ARG
    ix.inject_stall(0)
    q = W.P[W.query_idx[0]]
    assert np.array_equal(ix.rkmips(q, 10), oracle.rkmips(W.U, W.P, q, 10))
    ix.close()
