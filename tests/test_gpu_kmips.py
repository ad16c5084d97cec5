"""Standalone kMIPS through the SimHash tables (sah_kmips): SA-ALSH (SAT, Eq. 6-7) and
H2-ALSH's QNF (Eq. 3-4) over the same partitions, the paper's kMIPS comparison.

Pins: (1) where C covers every item (|P'| = n, or the probe radius at code_bits) the answer
is the exact top-k, up to items whose FP64 scores tie the k-th within FP32 rounding; (2)
with the same SRP matrix the answers equal the oracle's step-by-step loop for at least 90%
of the queries (an SRP sign or a stop test within rounding of zero may differ in FP32),
and every answer is well formed: distinct ids, descending scores equal to the FP64 score
within FP32 rounding, the seed P' never beaten by a left-out seed item."""
import numpy as np
import pytest

from oracle import sah as ref
import workload

pytestmark = pytest.mark.gpu


def _exact_topk_ok(P64, u, ids, k, rel=1e-5):
    sc = P64 @ u
    order = np.argsort(-sc, kind="stable")
    kth = sc[order[k - 1]]
    tol = rel * np.linalg.norm(u) * np.linalg.norm(P64, axis=1).max()
    assert len(ids) == k and len(set(ids.tolist())) == k
    assert np.all(sc[ids] >= kth - tol)                       # nothing below the k-th
    must = np.flatnonzero(sc > kth + tol)
    assert set(must.tolist()) <= set(ids.tolist())            # everything clearly above


def _index(sah, W, **kw):
    return sah.Index(W.U, W.P, k_max=50, leaf_size=32, **kw)


@pytest.mark.parametrize("transform", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_full_cover_is_exact_topk(sah, transform, precision):
    W = workload.make("c2", m=400, n=3000)
    P64 = W.P.astype(np.float64)
    Qu = W.U[:40]
    # |P'| = n: no partitions, C = every item
    ix = _index(sah, W, p_prime=1 << 30, precision=precision, transform=transform)
    for k in (1, 10, 50, 64):
        ids, sc = ix.kmips(Qu, k)
        for r in range(len(Qu)):
            _exact_topk_ok(P64, Qu[r].astype(np.float64), ids[r], k)
    ix.close()
    # the paper's |P'| with a full probe of 4-bit codes: every visited partition's items
    ix = _index(sah, W, p_prime=0, n_tables=6, code_bits=4, probe_radius=4, precision=precision,
                transform=transform)
    for k in (1, 10, 50):
        ids, sc = ix.kmips(Qu, k)
        for r in range(len(Qu)):
            u = Qu[r].astype(np.float64)
            _exact_topk_ok(P64, u, ids[r], k)
            assert np.allclose(sc[r], P64[ids[r]] @ u, rtol=1e-4, atol=1e-5 * np.linalg.norm(u) * 10)
    assert ix.stats()["n_partitions"] >= 2
    ix.close()


@pytest.mark.parametrize("transform,name", [(0, "sat"), (1, "qnf")])
@pytest.mark.parametrize("radius", [0, 1])
def test_equals_oracle_loop(sah, transform, name, radius):
    W = workload.make("c2", m=60, n=2500)
    K, bits = 8, 6
    A = workload.srp_matrix(K * bits, W.d + 1, seed=5)
    ix = _index(sah, W, p_prime=40, n_tables=K, code_bits=bits, probe_radius=radius, srp_matrix=A,
                precision=0, transform=transform)
    rix = ref.sah_index(W.P, W.U, kmax=50, N0=32, p_prime=40, A=A.astype(np.float64), n_tables=K,
                        code_bits=bits, b=0.5, transform=name)
    Qu = workload.make("c2", m=200, n=10, seed=3).U      # query vectors drawn like users
    P64 = W.P.astype(np.float64)
    same, total = 0, 0
    for k in (1, 10, 30):
        ids, sc = ix.kmips(Qu, k)
        for r in range(len(Qu)):
            u = Qu[r].astype(np.float64)
            want = rix.order[ref.sa_alsh_kmips(rix.saalsh, rix.P_sorted, u, k, np.arange(rix.p_prime), radius)]
            got = ids[r][ids[r] >= 0]
            # well formed: distinct, descending, scores equal to FP64 within FP32 rounding
            assert len(set(got.tolist())) == len(got)
            s64 = P64[got] @ u
            tol = 1e-5 * np.linalg.norm(u) * np.linalg.norm(P64, axis=1).max()
            assert np.all(np.abs(sc[r][:len(got)] - s64) <= tol)
            assert np.all(np.diff(sc[r][:len(got)]) <= 0)
            # the seed P' (the 40 largest norms) is always in C
            seed = rix.order[:40]
            if len(got) == k:
                left = np.setdiff1d(seed, got)
                assert np.all(P64[left] @ u <= s64[-1] + tol)
            same += int(set(got.tolist()) == set(want.tolist()))
            total += 1
    assert same >= 0.9 * total, (same, total)
    assert ix.stats()["items_scanned"] > 0
    ix.close()


def test_qnf_and_sat_differ_and_both_recall(sah):
    """Same partitions and tables, only the transform differs: the candidates scored differ,
    and SAT finds most of the exact top-10 at radius 1 with 64 tables of 8 bits."""
    W = workload.make("c2", m=60, n=6000)
    P64 = W.P.astype(np.float64)
    Qu = workload.make("c2", m=100, n=10, seed=4).U
    rec = {}
    scanned = {}
    for tr in (0, 1):
        ix = _index(sah, W, p_prime=0, n_tables=64, code_bits=8, probe_radius=1, precision=0, transform=tr)
        ids, _ = ix.kmips(Qu, 10)
        scanned[tr] = ix.stats()["items_scanned"]
        hits = 0
        for r in range(len(Qu)):
            sc = P64 @ Qu[r].astype(np.float64)
            truth = set(np.argsort(-sc, kind="stable")[:10].tolist())
            hits += len(truth & set(ids[r].tolist()))
        rec[tr] = hits / (10 * len(Qu))
        ix.close()
    assert scanned[0] != scanned[1]
    assert rec[0] > 0.5


def test_kmips_errors_and_device_buffers(sah):
    import torch
    W = workload.make("c1", m=100, n=500)
    ix = _index(sah, W, p_prime=0, n_tables=8, code_bits=6)
    for k in (0, 65):
        with pytest.raises(sah.SahError) as e:
            ix.kmips(W.U[:3], k)
        assert e.value.status == sah.SAH_ERR_ARG
    bad = W.U[:3].copy()
    bad[1, 2] = np.nan
    with pytest.raises(sah.SahError) as e:
        ix.kmips(bad, 5)
    assert e.value.status == sah.SAH_ERR_ARG
    ids_h, sc_h = ix.kmips(W.U[:7], 5)
    Qd = torch.from_numpy(W.U[:7]).cuda()
    ids_d = torch.empty((7, 5), dtype=torch.int32, device="cuda")
    sc_d = torch.empty((7, 5), dtype=torch.float32, device="cuda")
    ix.kmips_device(Qd, 5, ids_d, sc_d)
    torch.cuda.synchronize()
    assert np.array_equal(ids_d.cpu().numpy(), ids_h) and np.array_equal(sc_d.cpu().numpy(), sc_h)
    e_ids, _ = ix.kmips(np.zeros((0, W.d), np.float32), 5)
    assert e_ids.shape == (0, 5)
    ix.close()
