"""The continuous-batching server: every request's answer is the same as the blocking
call's for it alone, whatever batch it lands in; admission and slots behave."""
import time

import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu


def _drain(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_results_same_alone_and_in_the_mix(sah, precision):
    W = workload.make("c2", m=20000, n=3000)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=0, precision=precision, n_tables=16, code_bits=8)
    rng = np.random.default_rng(0)
    nreq = 300
    qi = rng.integers(0, W.n, nreq)
    ks = rng.integers(1, 51, nreq).astype(np.int32)
    modes = rng.integers(0, 2, nreq).astype(np.int32)
    alone = [ix.rkmips(W.P[qi[r]], ks[r], mode=int(modes[r])) for r in range(nreq)]
    srv = sah.Server(ix, max_slots=nreq, max_batch=64, workers=2)
    tickets = []
    for r in range(nreq):                      # bursts, so batches of many sizes form
        tickets.append(srv.submit(W.P[qi[r]], int(ks[r]), int(modes[r])))
        if r % 37 == 0:
            time.sleep(0.002)
    got = _drain(srv, tickets)
    for r, t in enumerate(tickets):
        ids, lat = got[t]
        assert np.array_equal(ids, alone[r]), r
        assert lat > 0
    info = srv.info()
    srv.stop()
    assert info["batched_requests"] == nreq and info["batches"] >= 2


def test_slots_budget_and_errors(sah):
    W = workload.make("c1", m=3000, n=800)
    ix = sah.Index(W.U, W.P, k_max=20, leaf_size=64)
    # a tiny budget forces every tick to shrink to single requests
    srv = sah.Server(ix, max_slots=8, max_batch=8, workers=1, hbm_budget_bytes=1)
    tickets = [srv.submit(W.P[i], 5) for i in range(8)]
    assert srv.try_submit(W.P[9], 5) is None                # every slot is taken
    got = _drain(srv, tickets)
    for i, t in enumerate(tickets):
        assert np.array_equal(got[t][0], ix.rkmips(W.P[i], 5))
    assert srv.info()["max_batch_seen"] == 1 and srv.info()["split_ticks"] > 0
    with pytest.raises(sah.SahError):
        srv.poll(123456)                                     # unknown ticket
    with pytest.raises(sah.SahError):
        srv.submit(W.P[0], 0)                                # k < 1
    srv.stop()


def test_repeated_batch_shapes_across_buffer_growth(sah):
    """Workers replay captured graphs for repeated batch shapes; batches that grow the
    worker's buffers in between (a larger workspace, more results) must not replay a graph
    captured against the freed ones.  Waves of 1, 7, 64, 7 and 1 requests, three times, each
    wave drained before the next, so that the same shapes recur after every growth."""
    W = workload.make("c2", m=20000, n=3000)
    ix = sah.Index(W.U, W.P, k_max=50, leaf_size=128, p_prime=0, precision=1, n_tables=16, code_bits=8)
    rng = np.random.default_rng(3)
    srv = sah.Server(ix, max_slots=256, max_batch=64, workers=1)
    checked = 0
    reqs = []
    for rep in range(3):
        for size in (1, 7, 64, 7, 1):
            qi = rng.integers(0, W.n, size)
            ks = rng.integers(1, 51, size)
            if rep == 2:
                ks[:] = 50                      # more answers: the result buffer grows
            tickets = [srv.submit(W.P[qi[r]], int(ks[r]), 0) for r in range(size)]
            got = _drain(srv, tickets)
            reqs += [(W.P[qi[r]], int(ks[r]), got[t][0]) for r, t in enumerate(tickets)]
    srv.stop()
    for q, k, ids in reqs:
        assert np.array_equal(ids, ix.rkmips(q, k))
        checked += 1
    assert checked == 3 * (1 + 7 + 64 + 7 + 1)
    ix.close()
