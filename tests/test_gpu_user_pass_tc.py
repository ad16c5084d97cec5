"""Tensor-core user pass (split BF16 operands on tcgen05, one persistent kernel per up to
256 queries): parity with the FP64 oracle on the shapes that exercise its tiling.

- more queries than one launch holds, with a ragged last launch and a query count that is
  not a multiple of 32 (the kept-pair bit words);
- fewer users than one 128-row tile, and a ragged last tile;
- leaves far smaller than a warp (many leaves per epilogue warp) and larger than a tile;
- d on both sides of 64 (one or two K-blocks per operand part);
- zero and duplicated users, k beyond k_max and beyond n, mixed modes, device buffers.
The bar is bit-exact for exact-mode rows."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

TC = dict(precision=1, tc_user_pass=1)


def _check(U, P, Q, K, got, rows):
    """rows[j] names the distinct query of row j; one oracle count answers every k."""
    counts = {}
    for j in range(len(K)):
        key = int(rows[j])
        if key not in counts:
            counts[key] = oracle.count_above(U, P, Q[j])
        want = np.flatnonzero(counts[key] < K[j]).astype(np.int32)
        assert np.array_equal(got[j], want), (j, int(K[j]))


@pytest.mark.parametrize("p_prime", [10, 1 << 30])
@pytest.mark.parametrize("d,nq", [(50, 300), (50, 256), (64, 257), (100, 300), (128, 129)])
def test_ragged_query_launches(sah, d, nq, p_prime):
    W = workload.make("c2", m=4000, n=1200, d=d)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=p_prime, **TC)
    rng = np.random.default_rng(d * 1000 + nq)
    distinct = rng.integers(0, W.n, 30)
    rows = distinct[rng.integers(0, len(distinct), nq)]
    K = rng.integers(1, 60, nq).astype(np.int32)           # k beyond k_max = 50 included
    K[::37] = W.n + 1                                        # every user
    Q = W.P[rows]
    got = ix.rkmips_batch(Q, K)
    _check(W.U, W.P, Q, K, got, rows)
    assert ix.stats()["users_scored"] > 0


@pytest.mark.parametrize("m", [1, 100, 128, 129, 300])
@pytest.mark.parametrize("leaf", [1, 4, 256])
def test_small_user_sets_and_leaves(sah, m, leaf):
    W = workload.make("c2", m=m, n=400, d=50)
    ix = sah.Index(W.U, W.P, k_max=20, leaf_size=leaf, p_prime=1 << 30, **TC)
    rows = np.repeat(W.query_idx[:6], 4)
    K = np.tile(np.array([1, 7, 20, 25], np.int32), 6)
    Q = W.P[rows]
    _check(W.U, W.P, Q, K, ix.rkmips_batch(Q, K), rows)


def test_zero_and_duplicate_users(sah):
    W = workload.make("c2", m=2000, n=700, d=50)
    U = W.U.copy()
    U[[0, 5, 1999]] = 0.0
    U[100:140] = U[7]
    ix = sah.Index(U, W.P, k_max=30, leaf_size=16, p_prime=1 << 30, **TC)
    rows = np.repeat(W.query_idx[:5], 3)
    K = np.tile(np.array([1, 30, 31], np.int32), 5)
    Q = W.P[rows]
    _check(U, W.P, Q, K, ix.rkmips_batch(Q, K), rows)


def test_same_answers_as_fp32_user_pass(sah):
    """The two user passes differ in arithmetic only: every exact-mode answer and the
    SA-ALSH answers agree, row by row."""
    W = workload.make("c2", m=6000, n=1500, d=50)
    A = workload.srp_matrix(8 * 6, W.d + 1, seed=5)
    kw = dict(k_max=50, leaf_size=64, p_prime=200, n_tables=8, code_bits=6, srp_matrix=A, seed=3)
    a = sah.Index(W.U, W.P, precision=1, tc_user_pass=0, **kw)
    b = sah.Index(W.U, W.P, precision=1, tc_user_pass=1, **kw)
    rows = np.repeat(W.query_idx[:20], 3)
    K = np.tile(np.array([3, 17, 50], np.int32), 20)
    modes = np.tile(np.array([sah.EXACT, sah.SAALSH], np.int32), 30)
    Q = W.P[rows]
    ga = a.rkmips_batch(Q, K, modes=modes)
    gb = b.rkmips_batch(Q, K, modes=modes)
    agree = total = 0
    for j in range(len(K)):
        if modes[j] == sah.EXACT:
            assert np.array_equal(ga[j], gb[j]), j
        else:
            sa, sb = set(ga[j].tolist()), set(gb[j].tolist())
            agree += len(sa & sb)
            total += len(sa | sb)
    assert total == 0 or agree / total >= 0.99
    _check(W.U, W.P, Q[modes == sah.EXACT], K[modes == sah.EXACT],
           [g for g, md in zip(gb, modes) if md == sah.EXACT], rows[modes == sah.EXACT])


def test_device_buffers(sah):
    import torch
    W = workload.make("c2", m=3000, n=1500, d=50)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=64, p_prime=1 << 30, **TC)
    Q, K, _ = W.requests()
    Q, K = Q[:270], K[:270]
    host = ix.rkmips_batch(Q, K)
    out = torch.empty(W.m * len(K), dtype=torch.int32, device="cuda")
    offs = torch.empty(len(K) + 1, dtype=torch.int64, device="cuda")
    total = ix.rkmips_batch_device(torch.from_numpy(Q).cuda(), torch.from_numpy(K).cuda(), out, offs)
    o = offs.cpu().numpy()
    res = out[:total].cpu().numpy()
    for j in range(len(K)):
        assert np.array_equal(res[o[j]:o[j + 1]], host[j])
