"""The answer bitmaps stay correct across calls (the compaction pass clears what it reads,
so the next call starts from zero): after a failed call, when the batch grows or shrinks,
with rows that ask for every user (k > n), and on the paper's |P'| with the two-phase
tensor-core kMIPS decision.  Every answer is checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

VARIANTS = {
    "fp32": dict(precision=0),
    "bf16-tc": dict(precision=1, tc_user_pass=1),
}


def _truth(U, P, q, k):
    return np.flatnonzero(oracle.count_above(U, P, q) < k).astype(np.int32)


def _check(W, Q, K, got):
    assert len(got) == len(K)
    for i, (q, k) in enumerate(zip(Q, K)):
        assert np.array_equal(got[i], _truth(W.U, W.P, q, int(k))), (i, int(k))


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_batch_sizes_grow_and_shrink(sah, variant):
    W = workload.make("c1", m=900, n=700)
    ix = sah.Index(W.U, W.P, k_max=20, leaf_size=16, p_prime=0, **VARIANTS[variant])
    rng = np.random.default_rng(3)
    for size in (3, 40, 1, 40, 17):
        rows = rng.integers(0, W.n, size)
        Q = np.ascontiguousarray(W.P[rows])
        K = rng.integers(1, 30, size).astype(np.int32)
        _check(W, Q, K, ix.rkmips_batch(Q, K))


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_after_buffer_too_small(sah, variant):
    W = workload.make("c1", m=800, n=500)
    ix = sah.Index(W.U, W.P, k_max=20, leaf_size=16, p_prime=0, **VARIANTS[variant])
    Q = np.ascontiguousarray(W.P[W.query_idx[:6]])
    K = np.array([1, 3, 5, 8, 13, 20], np.int32)
    with pytest.raises(sah.SahError) as e:
        ix.rkmips_batch(Q, K, cap=2)
    assert e.value.status == sah.SAH_ERR_BUFFER_TOO_SMALL
    # the next calls (the same batch, then another) see no answer of the failed one
    _check(W, Q, K, ix.rkmips_batch(Q, K))
    Q2 = np.ascontiguousarray(W.P[W.query_idx[6:9]])
    K2 = np.array([2, 4, 6], np.int32)
    _check(W, Q2, K2, ix.rkmips_batch(Q2, K2))


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_rows_asking_for_every_user(sah, variant):
    W = workload.make("c1", m=700, n=300)
    ix = sah.Index(W.U, W.P, k_max=20, leaf_size=16, p_prime=0, **VARIANTS[variant])
    Q = np.ascontiguousarray(W.P[W.query_idx[:4]])
    K = np.array([W.n + 1, 5, W.n + 7, 1], np.int32)
    got = ix.rkmips_batch(Q, K)
    assert np.array_equal(got[0], np.arange(W.m, dtype=np.int32))
    _check(W, Q, K, got)
    # a batch without such rows right after
    K2 = np.array([2, 3, 4, 9], np.int32)
    _check(W, Q, K2, ix.rkmips_batch(Q, K2))


def test_two_phase_decision_device_buffers(sah):
    """More than eight item tiles with the paper's |P'|: the tensor-core kMIPS decision
    runs its two scan phases; device buffers, the same batch three times (the last two
    replayed from a captured graph), then a different batch."""
    torch = pytest.importorskip("torch")
    W = workload.make("c2", m=5000, n=3000)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=64, p_prime=0, seed=2, precision=1, tc_user_pass=1)
    dev = torch.device("cuda", 0)
    qidx = W.query_idx[:10]
    Q = np.ascontiguousarray(np.repeat(W.P[qidx], 3, axis=0))
    K = np.tile(np.array([1, 10, 50], np.int32), len(qidx))
    host = ix.rkmips_batch(Q, K)
    _check(W, Q, K, host)
    total = sum(len(h) for h in host)
    Qd, Kd = torch.from_numpy(Q).to(dev), torch.from_numpy(K).to(dev)
    out = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    offs = torch.empty(len(K) + 1, dtype=torch.int64, device=dev)
    for _ in range(3):
        ix.rkmips_batch_device(Qd, Kd, out, offs)
        torch.cuda.synchronize()
        o = offs.cpu().numpy()
        ids = out.cpu().numpy()
        for i in range(len(K)):
            assert np.array_equal(ids[o[i]:o[i + 1]], host[i]), i
    Q2 = np.ascontiguousarray(W.P[W.query_idx[10:14]])
    K2 = np.array([3, 7, 20, 40], np.int32)
    _check(W, Q2, K2, ix.rkmips_batch(Q2, K2))
