"""Batch calls on pinned host buffers, which the kernels read and write in place (one
synchronisation, no staging copy): the answers equal those of the same call on pageable
host buffers and the FP64 oracle's; a too-small buffer and an invalid k report as on the
other paths; a pageable output beside pinned inputs takes the copying path."""
import ctypes

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def _pinned(a):
    torch = pytest.importorskip("torch")
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _call(ix, Q, K, out, offs, modes=None):
    return ix.raw_batch(Q.data_ptr(), Q.shape[0], K.data_ptr(), modes.data_ptr() if modes is not None else None, 0,
                        out.data_ptr(), out.numel(), offs.data_ptr())


@pytest.mark.parametrize("precision,tc", [(0, 0), (1, 1)])
def test_pinned_buffers_match_pageable_and_oracle(sah, precision, tc):
    torch = pytest.importorskip("torch")
    W = workload.make("c1", m=1500, n=900)
    ix = sah.Index(W.U, W.P, k_max=20, leaf_size=32, p_prime=0, precision=precision, tc_user_pass=tc)
    rows = W.query_idx[:12]
    Q = np.ascontiguousarray(np.repeat(W.P[rows], 2, axis=0))
    K = np.tile(np.array([3, 17], np.int32), len(rows))
    ref = ix.rkmips_batch(Q, K)
    total = sum(len(r) for r in ref)
    Qp, Kp = _pinned(Q), _pinned(K)
    out = torch.empty(total + 5, dtype=torch.int32).pin_memory()
    offs = torch.empty(len(K) + 1, dtype=torch.int64).pin_memory()
    for _ in range(3):   # the later calls replay the captured graph
        out.fill_(-1)
        assert _call(ix, Qp, Kp, out, offs) == 0
        o = offs.numpy()
        assert o[-1] == total
        for i in range(len(K)):
            got = out.numpy()[o[i]:o[i + 1]]
            assert np.array_equal(got, ref[i]), i
            want = np.flatnonzero(oracle.count_above(W.U, W.P, Q[i]) < K[i]).astype(np.int32)
            assert np.array_equal(got, want), i


def test_pinned_too_small_and_invalid_k(sah):
    torch = pytest.importorskip("torch")
    W = workload.make("c1", m=800, n=500)
    ix = sah.Index(W.U, W.P, k_max=20, leaf_size=16, p_prime=0, precision=1, tc_user_pass=1)
    Q = np.ascontiguousarray(W.P[W.query_idx[:4]])
    K = np.array([5, 9, 13, 20], np.int32)
    ref = ix.rkmips_batch(Q, K)
    need = sum(len(r) for r in ref)
    Qp, Kp = _pinned(Q), _pinned(K)
    small = torch.empty(max(need - 1, 1), dtype=torch.int32).pin_memory()
    offs = torch.zeros(len(K) + 1, dtype=torch.int64).pin_memory()
    assert _call(ix, Qp, Kp, small, offs) == sah.SAH_ERR_BUFFER_TOO_SMALL
    assert offs.numpy()[-1] == need
    assert np.array_equal(np.diff(offs.numpy()), [len(r) for r in ref])
    bad = _pinned(np.array([5, 0, 13, 20], np.int32))
    big = torch.empty(need, dtype=torch.int32).pin_memory()
    assert _call(ix, Qp, bad, big, offs) == sah.SAH_ERR_ARG
    # the next call on the same buffers is unaffected
    assert _call(ix, Qp, Kp, big, offs) == 0
    o = offs.numpy()
    for i in range(len(K)):
        assert np.array_equal(big.numpy()[o[i]:o[i + 1]], ref[i])


def test_pinned_inputs_pageable_output(sah):
    torch = pytest.importorskip("torch")
    W = workload.make("c1", m=700, n=400)
    ix = sah.Index(W.U, W.P, k_max=10, leaf_size=16, p_prime=0)
    Q = np.ascontiguousarray(W.P[W.query_idx[:3]])
    K = np.array([1, 4, 10], np.int32)
    ref = ix.rkmips_batch(Q, K)
    Qp, Kp = _pinned(Q), _pinned(K)
    out = np.empty(sum(len(r) for r in ref) + 1, np.int32)
    offs = np.empty(len(K) + 1, np.int64)
    st = ix.raw_batch(Qp.data_ptr(), 3, Kp.data_ptr(), None, 0, out.ctypes.data, out.size, offs.ctypes.data)
    assert st == 0
    for i in range(3):
        assert np.array_equal(out[offs[i]:offs[i + 1]], ref[i])


def test_pinned_two_sub_batches(sah):
    """More rows than one sub-batch holds (4096): the answers gather in the library's
    buffer and are copied into the pinned output at the end."""
    torch = pytest.importorskip("torch")
    W = workload.make("c1", m=700, n=400)
    ix = sah.Index(W.U, W.P, k_max=10, leaf_size=16, p_prime=0, precision=1, tc_user_pass=1)
    rng = np.random.default_rng(11)
    nq = 4500
    Q = np.ascontiguousarray(W.P[rng.integers(0, W.n, nq)])
    K = rng.integers(1, 13, nq).astype(np.int32)
    ref = ix.rkmips_batch(Q, K)
    total = sum(len(r) for r in ref)
    Qp, Kp = _pinned(Q), _pinned(K)
    out = torch.empty(max(total, 1), dtype=torch.int32).pin_memory()
    offs = torch.empty(nq + 1, dtype=torch.int64).pin_memory()
    assert _call(ix, Qp, Kp, out, offs) == 0
    o = offs.numpy()
    assert o[-1] == total
    for i in range(nq):
        assert np.array_equal(out.numpy()[o[i]:o[i + 1]], ref[i]), i
    for i in range(0, nq, 450):
        want = np.flatnonzero(oracle.count_above(W.U, W.P, Q[i]) < K[i]).astype(np.int32)
        assert np.array_equal(out.numpy()[o[i]:o[i + 1]], want), i


def test_pinned_mixed_modes(sah):
    """Pinned requests with a pinned modes array (half the rows in SA-ALSH mode): the same
    answers as the call on pageable buffers; the exact rows equal the oracle's."""
    torch = pytest.importorskip("torch")
    W = workload.make("c1", m=1200, n=800)
    ix = sah.Index(W.U, W.P, k_max=20, leaf_size=32, p_prime=0, precision=1, tc_user_pass=1, n_tables=16,
                   code_bits=8)
    rows = W.query_idx[:10]
    Q = np.ascontiguousarray(np.repeat(W.P[rows], 2, axis=0))
    K = np.tile(np.array([4, 15], np.int32), len(rows))
    modes = np.tile(np.array([sah.SAALSH, sah.EXACT], np.int32), len(rows))
    ref = ix.rkmips_batch(Q, K, modes=modes)
    Qp, Kp, Mp = _pinned(Q), _pinned(K), _pinned(modes)
    out = torch.empty(sum(len(r) for r in ref) + 1, dtype=torch.int32).pin_memory()
    offs = torch.empty(len(K) + 1, dtype=torch.int64).pin_memory()
    assert _call(ix, Qp, Kp, out, offs, modes=Mp) == 0
    o = offs.numpy()
    for i in range(len(K)):
        got = out.numpy()[o[i]:o[i + 1]]
        assert np.array_equal(got, ref[i]), i
        if modes[i] == sah.EXACT:
            want = np.flatnonzero(oracle.count_above(W.U, W.P, Q[i]) < K[i]).astype(np.int32)
            assert np.array_equal(got, want), i
