"""Exact-mode parity of the CUDA path (through the C-ABI) with the FP64 oracle.

The bar is bit-exact: result sets are integer data, and the exact mode decides every
user the FP32 error bound leaves open in the oracle's own double-precision order, so
the sets must be identical, near-ties included (no margin exclusion).
"""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


# precision variants: FP32 on the CUDA cores; BF16 copies with the FP32 user pass; BF16
# copies with the tensor-core user pass (BF16 operands); the tensor-core user pass on E4M3
# operands with per-vector scales (a band of about 0.13 ||u|| ||q||, most pairs re-scored)
VARIANTS = {
    "fp32": dict(precision=0),
    "bf16-simt": dict(precision=1, tc_user_pass=0),
    "bf16-tc": dict(precision=1, tc_user_pass=1),
    "fp8-tc": dict(precision=1, tc_user_pass=2),
}


def _truth(U, P, q, ks):
    c = oracle.count_above(U, P, q)
    return {int(k): np.flatnonzero(c < k).astype(np.int32) for k in ks}


def test_c1_every_query_and_k(sah):
    W = workload.make("c1")
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=20)
    ks = (1, 5, 10, 50, 51, 200, W.n, W.n + 1)
    for qi in W.query_idx:
        q = W.P[qi]
        want = _truth(W.U, W.P, q, ks)
        for k in ks:
            assert np.array_equal(ix.rkmips(q, k), want[k]), (qi, k)


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("leaf", [1, 20, 256])
@pytest.mark.parametrize("p_prime", [10, 0, 1 << 30])      # small P', 4 k_max, all items
def test_mf_batch_mixed_k(sah, leaf, p_prime, variant):
    W = workload.make("c2", m=6000, n=2500)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=leaf, p_prime=p_prime, seed=7, **VARIANTS[variant])
    ks = [1, 5, 10, 20, 50, 64]
    qidx = W.query_idx[:8]
    Q = np.repeat(W.P[qidx], len(ks), axis=0)
    K = np.tile(np.array(ks, np.int32), len(qidx))
    got = ix.rkmips_batch(Q, K)
    for a, qi in enumerate(qidx):
        want = _truth(W.U, W.P, W.P[qi], ks)
        for b, k in enumerate(ks):
            assert np.array_equal(got[a * len(ks) + b], want[k]), (qi, k, leaf, p_prime)
    st = ix.stats()
    assert st["queries"] == len(Q) and st["results"] == sum(len(g) for g in got)


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("seed", range(4))
def test_integer_ties(sah, seed, variant):
    P, U, q = workload.tie_case(40, 300, 3, lo=-2, hi=2, seed=seed)
    ix = sah.Index(U, P, k_max=8, leaf_size=4, p_prime=6, seed=seed, **VARIANTS[variant])
    for qq in (q, P[seed]):                                         # q outside and inside P
        want = _truth(U, P, qq, range(1, 42))
        for k in range(1, 42):
            assert np.array_equal(ix.rkmips(qq, k), want[k]), (seed, k)


def test_zero_duplicate_users_and_items(sah):
    W = workload.make("c1", m=500, n=300)
    U = W.U.copy()
    U[[0, 7, 499]] = 0.0
    U[10:20] = U[30]                                                # duplicated users
    P = np.vstack([W.P, W.P[:5]])                                  # duplicated items
    ix = sah.Index(U, P, k_max=20, leaf_size=8)
    for qi in W.query_idx[:5]:
        q = P[qi]
        want = _truth(U, P, q, (1, 3, 20, 25))
        for k in (1, 3, 20, 25):
            assert np.array_equal(ix.rkmips(q, k), want[k])


def test_zero_query_and_foreign_query(sah):
    W = workload.make("c1", m=400, n=200)
    ix = sah.Index(W.U, W.P, k_max=16, leaf_size=16)
    rng = np.random.default_rng(4)
    for q in (np.zeros(W.d, np.float32), rng.standard_normal(W.d).astype(np.float32) * 3):
        want = _truth(W.U, W.P, q, (1, 10, 16, 17, W.n, W.n + 1))
        for k in want:
            assert np.array_equal(ix.rkmips(q, k), want[k])


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("d", [1, 3, 50, 64, 65, 100, 128, 300])
def test_dimensions(sah, d, variant):
    W = workload.make("c1", m=700, n=600, d=d)
    kw = VARIANTS[variant]
    if kw["precision"] == 1 and d > 128:
        with pytest.raises(sah.SahError) as e:
            sah.Index(W.U, W.P, k_max=10, leaf_size=32, **kw)
        assert e.value.status == sah.SAH_ERR_UNSUPPORTED
        return
    ix = sah.Index(W.U, W.P, k_max=10, leaf_size=32, p_prime=12, **kw)
    for qi in W.query_idx[:3]:
        q = W.P[qi]
        want = _truth(W.U, W.P, q, (1, 10, 11))
        for k in want:
            assert np.array_equal(ix.rkmips(q, k), want[k]), (d, k)


def test_single_user_single_item(sah):
    U = np.array([[1.0, 2.0]], np.float32)
    P = np.array([[0.5, -1.0]], np.float32)
    ix = sah.Index(U, P, k_max=1, leaf_size=1)
    assert ix.rkmips(P[0], 1).tolist() == [0]
    assert ix.rkmips(np.array([-5.0, 0.0], np.float32), 1).tolist() == []
    assert ix.rkmips(np.array([-5.0, 0.0], np.float32), 2).tolist() == [0]


def test_device_buffers_match_host_buffers(sah):
    import torch
    W = workload.make("c2", m=3000, n=1500)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=64)
    Q, K, _ = workload.make("c2", m=3000, n=1500).requests()
    Q, K = Q[:60], K[:60]
    host = ix.rkmips_batch(Q, K)
    Qd = torch.from_numpy(Q).cuda()
    Kd = torch.from_numpy(K).cuda()
    out = torch.empty(W.m * len(K), dtype=torch.int32, device="cuda")
    offs = torch.empty(len(K) + 1, dtype=torch.int64, device="cuda")
    total = ix.rkmips_batch_device(Qd, Kd, out, offs)
    o = offs.cpu().numpy()
    res = out[:total].cpu().numpy()
    for j in range(len(K)):
        assert np.array_equal(res[o[j]:o[j + 1]], host[j])


def test_index_from_device_inputs(sah):
    import torch
    W = workload.make("c1", m=800, n=500)
    a = sah.Index(W.U, W.P, k_max=10, leaf_size=20)
    b = sah.Index(torch.from_numpy(W.U).cuda(), torch.from_numpy(W.P).cuda(), k_max=10, leaf_size=20)
    q = W.P[W.query_idx[0]]
    for k in (1, 10):
        assert np.array_equal(a.rkmips(q, k), b.rkmips(q, k))


def test_errors_and_buffer_too_small(sah):
    W = workload.make("c1", m=300, n=200)
    ix = sah.Index(W.U, W.P, k_max=10, leaf_size=16)
    q = W.P[W.query_idx[0]]
    with pytest.raises(sah.SahError) as e:
        ix.rkmips(q, 0)
    assert e.value.status == sah.SAH_ERR_ARG
    bad = q.copy()
    bad[0] = np.nan
    with pytest.raises(sah.SahError) as e:
        ix.rkmips(bad, 3)
    assert e.value.status == sah.SAH_ERR_ARG
    want = _truth(W.U, W.P, q, (W.n + 1,))[W.n + 1]
    with pytest.raises(sah.SahError) as e:
        ix.rkmips_batch(q[None], [W.n + 1], cap=10)
    assert e.value.status == sah.SAH_ERR_BUFFER_TOO_SMALL
    # the index stays usable afterwards
    assert np.array_equal(ix.rkmips(q, W.n + 1), want)
    with pytest.raises(sah.SahError) as e:
        sah.Index(W.U, W.P, k_max=0)
    assert e.value.status == sah.SAH_ERR_ARG
    Ubad = W.U.copy()
    Ubad[3, 2] = np.inf
    with pytest.raises(sah.SahError) as e:
        sah.Index(Ubad, W.P)
    assert e.value.status == sah.SAH_ERR_ARG


def test_empty_batch(sah):
    W = workload.make("c1", m=100, n=100)
    ix = sah.Index(W.U, W.P, k_max=10, leaf_size=16)
    assert ix.rkmips_batch(np.zeros((0, W.d), np.float32), np.zeros(0, np.int32)) == []


@pytest.mark.slow
@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("p_prime", [0, 1 << 30])
def test_c2_full_size_sampled(sah, p_prime, variant):
    """n = 17,770, m = 480,000, d = 50 (the benchmark's workload): the answers of a fixed
    sample of users, plus every user the GPU returned, agree with the oracle."""
    W = workload.make("c2")
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=256, p_prime=p_prime, **VARIANTS[variant])
    ks = [int(k) for k in W.ks]
    qidx = W.query_idx[:6]
    Q = np.repeat(W.P[qidx], len(ks), axis=0)
    K = np.tile(np.array(ks, np.int32), len(qidx))
    got = ix.rkmips_batch(Q, K)
    sample = workload.sample_rows(W.m, 1500, seed=11)
    for a, qi in enumerate(qidx):
        returned = np.unique(np.concatenate([got[a * len(ks) + b] for b in range(len(ks))]))
        users = np.union1d(sample, returned[:3000])
        c = oracle.count_above(W.U, W.P, W.P[qi], users)
        for b, k in enumerate(ks):
            g = set(got[a * len(ks) + b].tolist())
            member = np.array([u in g for u in users.tolist()])
            assert np.array_equal(member, c < k), (qi, k)


def test_tensor_core_path_runs_and_counts(sah):
    """With BF16 the kMIPS decisions go through the tcgen05 kernel (several launches per
    call in the decision stage) and give the oracle's answers."""
    W = workload.make("c2", m=8000, n=3000)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=60, precision=sah.BF16)
    ix.set_timing(True)
    Q, K, _ = W.requests()
    Q, K = Q[:50], K[:50]
    got = ix.rkmips_batch(Q, K)
    st = ix.stats()
    assert st["survivors"] > 1000 and st["items_scanned"] > 0
    assert st["stage_launches"][3] >= 6
    for j in range(0, 50, 7):
        c = oracle.count_above(W.U, W.P, Q[j])
        assert np.array_equal(got[j], np.flatnonzero(c < K[j]))


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_survivor_list_overflow_reruns(sah, variant):
    """More survivors than the list's first capacity (64k): the call grows the list, runs
    the sub-batch again and still returns the oracle's answers."""
    W = workload.make("c2", m=20000, n=800)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=5, **VARIANTS[variant])
    rng = np.random.default_rng(3)
    rows = rng.integers(0, W.n, 200)
    Q = W.P[rows]
    K = np.full(200, 30, np.int32)
    got = ix.rkmips_batch(Q, K)
    assert ix.stats()["survivors"] > (1 << 16)
    for r in (0, 57, 123, 199):
        assert np.array_equal(got[r], _truth(W.U, W.P, Q[r], (30,))[30]), r


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_repeated_calls_same_answers(sah, variant):
    """A call whose shapes and buffers repeat is captured as a CUDA graph on its second run
    and replayed after that: every run, host or device buffers, interleaved with other
    shapes and with per-stage timing on and off, gives the oracle's answers."""
    import torch
    W = workload.make("c2", m=5000, n=1500)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=1 << 30, **VARIANTS[variant])
    Q, K, rows = W.requests()
    Q, K, rows = Q[:120], K[:120], rows[:120]
    counts = {int(r): oracle.count_above(W.U, W.P, W.P[W.query_idx[r]]) for r in np.unique(rows)}
    want = [np.flatnonzero(counts[int(rows[j])] < K[j]).astype(np.int32) for j in range(len(K))]
    Qd, Kd = torch.from_numpy(Q).cuda(), torch.from_numpy(K).cuda()
    out = torch.empty(W.m * len(K), dtype=torch.int32, device="cuda")
    offs = torch.empty(len(K) + 1, dtype=torch.int64, device="cuda")
    for it in range(6):
        ix.set_timing(it == 4)
        got = ix.rkmips_batch(Q, K)
        assert all(np.array_equal(g, w) for g, w in zip(got, want)), it
        total = ix.rkmips_batch_device(Qd, Kd, out, offs)
        o = offs.cpu().numpy()
        res = out[:total].cpu().numpy()
        assert all(np.array_equal(res[o[j]:o[j + 1]], want[j]) for j in range(len(K))), it
        small = ix.rkmips_batch(Q[:7], K[:7])                 # another shape in between
        assert all(np.array_equal(g, w) for g, w in zip(small, want[:7])), it


@pytest.mark.parametrize("variant", ["bf16-tc", "fp8-tc"])
@pytest.mark.parametrize("p_prime", [0, 1 << 30])
def test_sub_batch_past_shared_memory_column_table(sah, variant, p_prime):
    """9,000 rows in one call (one tensor-core sub-batch, whose column table no longer fits in
    shared memory: about 6,000 distinct vectors) give the answers of the same rows asked in
    calls of 700 rows, and a sample of rows agrees with the oracle."""
    W = workload.make("c2", m=6000, n=2500)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=p_prime, seed=3, **VARIANTS[variant])
    rng = np.random.default_rng(21)
    nrow = 9000
    # rows: items of P, foreign vectors and repeats of both, each with its own k
    foreign = (rng.standard_normal((3500, W.d)) * W.P.std()).astype(np.float32)
    pool = np.vstack([W.P, foreign])
    pick = rng.integers(0, len(pool), nrow)
    Q = pool[pick]
    K = rng.choice(np.array([1, 2, 5, 10, 25, 50, 51, 300], np.int32), nrow)
    whole = ix.rkmips_batch(Q, K)
    parts = []
    for a in range(0, nrow, 700):
        parts += ix.rkmips_batch(Q[a:a + 700], K[a:a + 700])
    for j in range(nrow):
        assert np.array_equal(whole[j], parts[j]), j
    for j in rng.choice(nrow, 24, replace=False):
        c = oracle.count_above(W.U, W.P, Q[j])
        assert np.array_equal(whole[j], np.flatnonzero(c < K[j]).astype(np.int32)), (j, int(K[j]))


@pytest.mark.parametrize("variant", ["bf16-tc", "fp8-tc"])
@pytest.mark.parametrize("nrows", [400, 2100])             # the one-CTA and the grid-wide build
def test_hash_collisions_rebuild_the_column_table(sah, variant, nrows):
    """Every row given one hash: the bitwise check finds the different vectors sharing a
    column and the table is built again comparing whole vectors, with unchanged answers."""
    W = workload.make("c2", m=5000, n=2000)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=1 << 30, seed=5, **VARIANTS[variant])
    rng = np.random.default_rng(8)
    vecs = W.P[rng.choice(W.n, 150, replace=False)]
    pick = rng.integers(0, 150, nrows)                     # 150 vectors, most asked several times
    Q = vecs[pick]
    K = rng.choice(np.array([1, 3, 10, 50, 60], np.int32), len(pick))
    plain = ix.rkmips_batch(Q, K)
    ix.inject_hash_collision(True)
    hooked = ix.rkmips_batch(Q, K)
    again = ix.rkmips_batch(Q, K)                          # the hook has cleared itself
    for j in range(len(K)):
        assert np.array_equal(plain[j], hooked[j]) and np.array_equal(plain[j], again[j]), j
    for j in rng.choice(len(K), 8, replace=False):
        c = oracle.count_above(W.U, W.P, Q[j])
        assert np.array_equal(plain[j], np.flatnonzero(c < K[j]).astype(np.int32)), j


def test_tensor_core_call_over_several_sub_batches(sah):
    """20,000 rows in one call take two sub-batches of the tensor-core path (16,384 + 3,616
    rows, the second built by the grid-wide column table): the answers equal those of the
    same rows asked in calls of 5,000, and a sample agrees with the oracle."""
    W = workload.make("c2", m=6000, n=2500)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=1 << 30, seed=4, **VARIANTS["bf16-tc"])
    rng = np.random.default_rng(33)
    nrow = 20000
    Q = W.P[rng.integers(0, W.n, nrow)]
    K = rng.choice(np.array([1, 5, 10, 50, 51, W.n + 1], np.int32), nrow)
    whole = ix.rkmips_batch(Q, K)
    parts = []
    for a in range(0, nrow, 5000):
        parts += ix.rkmips_batch(Q[a:a + 5000], K[a:a + 5000])
    for j in range(nrow):
        assert np.array_equal(whole[j], parts[j]), j
    for j in rng.choice(nrow, 16, replace=False):
        c = oracle.count_above(W.U, W.P, Q[j])
        assert np.array_equal(whole[j], np.flatnonzero(c < K[j]).astype(np.int32)), (j, int(K[j]))
