"""The allocation-free entry point against the FP64 oracle and the index-based exact path.

sah_rkmips_bruteforce_noalloc serves callers that may not allocate device memory on their
request path; its only scratch is a fixed array inside the library that every call shares.
This file is collected last so that a run stopping at its first failure has already run
every other test; it passes alone and after the others.
"""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def _run(sah, Ud, Pd, q, k, out, cnt):
    import torch
    sah.rkmips_bruteforce_noalloc(Ud, Pd, torch.from_numpy(np.ascontiguousarray(q)).cuda(), k, out, cnt)
    torch.cuda.synchronize()
    return int(cnt.item())


def test_noalloc_matches_index_path_on_two_calls_in_a_row(sah):
    import torch
    W = workload.make("c2", m=20000, n=1500)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=64)
    Ud = torch.from_numpy(W.U).cuda()
    Pd = torch.from_numpy(W.P).cuda()
    out = torch.full((W.m,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    norms = np.linalg.norm(W.P[W.query_idx], axis=1)
    big = W.query_idx[int(np.argmax(norms))]     # a 3x-norm item: a large answer first
    small = W.query_idx[int(np.argmin(norms))]   # then a small one: stale bits would show
    for qi, k in ((big, 50), (small, 1)):
        q = W.P[qi]
        want = ix.rkmips(q, k)
        c = _run(sah, Ud, Pd, q, k, out, cnt)
        assert c == len(want)
        assert np.array_equal(out[:c].cpu().numpy(), want)
        assert np.array_equal(want, oracle.rkmips(W.U, W.P, q, k))


def test_noalloc_equals_oracle_on_ragged_sizes_and_ties(sah):
    """m not a multiple of 32 (the last bitmap word partly used), against the FP64 oracle
    directly; and integer data where ties are frequent (every tie is settled in double
    precision, where it is exact)."""
    import torch
    W = workload.make("c2", m=1000, n=700)
    Ud, Pd = torch.from_numpy(W.U).cuda(), torch.from_numpy(W.P).cuda()
    out = torch.full((W.m,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for qi in W.query_idx[:4]:
        for k in (1, 7, 50, 700, 701):
            c = _run(sah, Ud, Pd, W.P[qi], k, out, cnt)
            assert np.array_equal(out[:c].cpu().numpy(), oracle.rkmips(W.U, W.P, W.P[qi], k)), (qi, k)
    P, U, q = workload.tie_case(40, 333, 3, seed=7)
    Ud, Pd = torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda()
    out = torch.full((333,), -1, dtype=torch.int32, device="cuda")
    for qq in (q, P[5]):
        for k in (1, 2, 5, 40, 41):
            c = _run(sah, Ud, Pd, qq, k, out, cnt)
            assert np.array_equal(out[:c].cpu().numpy(), oracle.rkmips(U, P, qq, k)), k


def test_noalloc_count_without_ids_when_cap_is_short(sah):
    """cap below the answer's size: *out_count holds the full size and no id is written."""
    import torch
    W = workload.make("c2", m=3000, n=500)
    Ud, Pd = torch.from_numpy(W.U).cuda(), torch.from_numpy(W.P).cuda()
    q = W.P[W.query_idx[0]]
    want = oracle.rkmips(W.U, W.P, q, 50)
    assert len(want) >= 2
    short = torch.full((len(want) - 1,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert _run(sah, Ud, Pd, q, 50, short, cnt) == len(want)
    assert bool((short == -1).all())
    exact = torch.full((len(want),), -1, dtype=torch.int32, device="cuda")
    assert _run(sah, Ud, Pd, q, 50, exact, cnt) == len(want)
    assert np.array_equal(exact.cpu().numpy(), want)


def test_noalloc_at_its_user_limit(sah):
    """m = 2^22 users, the largest the fixed scratch array holds (every bitmap word used)."""
    import torch
    m = sah.NOALLOC_MAX_USERS
    W = workload.make("c1", m=m, n=64, d=8)
    Ud, Pd = torch.from_numpy(W.U).cuda(), torch.from_numpy(W.P).cuda()
    out = torch.full((m,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    q = W.P[W.query_idx[0]]
    for k in (3, 1):
        c = _run(sah, Ud, Pd, q, k, out, cnt)
        assert np.array_equal(out[:c].cpu().numpy(), oracle.rkmips(W.U, W.P, q, k)), k


def test_noalloc_rejects_sizes_beyond_its_scratch(sah):
    import torch
    U = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(sah.SahError) as e:
        sah.rkmips_bruteforce_noalloc(U, U, U[0], 1, out, cnt, m=sah.NOALLOC_MAX_USERS + 1)
    assert e.value.status == sah.SAH_ERR_ARG


def test_noalloc_binding_rejects_mismatched_tensors(sah):
    """The binding checks dtype, layout, device and shapes before the call (it converts
    nothing, so it still allocates nothing)."""
    import torch
    U = torch.zeros((8, 3), dtype=torch.float32, device="cuda")
    out = torch.empty(8, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    bad_calls = [
        (U.double(), U, U[0], out, cnt),                 # float64 users
        (U.t(), U, U[0], out, cnt),                      # transposed (non-contiguous)
        (U, U[:, :2].contiguous(), U[0], out, cnt),      # P with another d
        (U, U, U[0, :2], out, cnt),                      # q of the wrong length
        (U, U, U[0], out.long(), cnt),                   # int64 ids
        (U, U, U[0], out, cnt.int()),                    # int32 count
        (U.cpu(), U, U[0], out, cnt),                    # a host tensor
    ]
    for args in bad_calls:
        with pytest.raises(sah.SahError) as e:
            sah.rkmips_bruteforce_noalloc(args[0], args[1], args[2], 1, args[3], args[4])
        assert e.value.status == sah.SAH_ERR_ARG
