"""The allocation-free entry point agrees with the index-based exact path.

sah_rkmips_bruteforce_noalloc serves callers that may not allocate device memory on their
request path; its only scratch is a fixed array inside the library that every call shares.
This file is collected last so that a run stopping at its first failure has already run
every other test; it passes alone and after the others.
"""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu


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
        sah.rkmips_bruteforce_noalloc(Ud, Pd, torch.from_numpy(q).cuda(), k, out, cnt)
        torch.cuda.synchronize()
        c = int(cnt.item())
        assert c == len(want)
        assert np.array_equal(out[:c].cpu().numpy(), want)


def test_noalloc_rejects_sizes_beyond_its_scratch(sah):
    import torch
    U = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(sah.SahError) as e:
        sah.rkmips_bruteforce_noalloc(U, U, U[0], 1, out, cnt, m=sah.NOALLOC_MAX_USERS + 1)
    assert e.value.status == sah.SAH_ERR_ARG
