"""SA-ALSH mode (Alg. 1, Alg. 2) of the CUDA path.

SA-ALSH is approximate by design (Thm. 2), so its parity with the oracle is pinned by
properties rather than bit equality: (1) every "no" is backed by k items that certainly
beat <u,q>, so the answer is a superset of the exact one; (2) probing every code
(probe radius = code_bits) makes every item a candidate and gives the exact answer; (3)
with the same SRP matrix it agrees with the oracle's step-by-step Alg. 2 except where an
SRP sign is within rounding of zero."""
import numpy as np
import pytest

import oracle
from oracle import sah as ref
import workload

pytestmark = pytest.mark.gpu


def _setup(sah, probe_radius=0, K=8, bits=6, m=1200, n=900, p_prime=40, precision=0, tc_user_pass=0):
    W = workload.make("c2", m=m, n=n)
    A = workload.srp_matrix(K * bits, W.d + 1, seed=5)
    ix = sah.Index(W.U, W.P, k_max=20, leaf_size=32, p_prime=p_prime, n_tables=K, code_bits=bits,
                   probe_radius=probe_radius, srp_matrix=A, precision=precision, tc_user_pass=tc_user_pass)
    return W, A, ix


@pytest.mark.parametrize("precision,tc", [(0, 0), (1, 0), (1, 1), (2, 1)])
def test_superset_of_exact_and_f1(sah, precision, tc):
    W, A, ix = _setup(sah, precision=precision, tc_user_pass=tc)
    f1s = []
    for qi in W.query_idx[:6]:
        q = W.P[qi]
        for k in (1, 5, 20):
            got = ix.rkmips(q, k, mode=sah.SAALSH)
            exact = oracle.rkmips(W.U, W.P, q, k)
            assert set(exact.tolist()) <= set(got.tolist())
            f1s.append(oracle.f1(got, exact))
    assert ix.stats()["n_partitions"] >= 2
    assert np.mean(f1s) > 0.5


@pytest.mark.parametrize("precision", [0, 2])
def test_full_probe_is_exact(sah, precision):
    W, A, ix = _setup(sah, probe_radius=6, precision=precision)
    for qi in W.query_idx[:4]:
        q = W.P[qi]
        for k in (1, 10, 20):
            assert np.array_equal(ix.rkmips(q, k, mode=sah.SAALSH), oracle.rkmips(W.U, W.P, q, k))


# FP32 codes; tensor-core codes with split BF16 and with FP8 E4M3 operands (more code bits
# fall on the other side of zero with FP8: a looser bar)
@pytest.mark.parametrize("precision,bar", [(0, 0.95), (1, 0.95), (2, 0.8)])
def test_agrees_with_oracle_alg2(sah, precision, bar):
    W, A, ix = _setup(sah, m=500, n=600, precision=precision)
    rix = ref.sah_index(W.P, W.U, kmax=20, N0=32, p_prime=40, A=A.astype(np.float64), n_tables=8,
                        code_bits=6, b=0.5)
    agree, total = 0, 0
    for qi in W.query_idx[:3]:
        q = W.P[qi]
        for k in (1, 10):
            got = set(ix.rkmips(q, k, mode=sah.SAALSH).tolist())
            want = set(ref.sah_query(rix, q, k, "saalsh", probe_radius=0).tolist())
            agree += len(got & want)
            total += len(got | want)
    assert total == 0 or agree / total >= bar


@pytest.mark.parametrize("precision,tc", [(0, 0), (1, 1), (2, 1)])
def test_mixed_modes_in_one_batch(sah, precision, tc):
    W, A, ix = _setup(sah, precision=precision, tc_user_pass=tc)
    Q = np.repeat(W.P[W.query_idx[:5]], 2, axis=0)
    K = np.array([10] * 10, np.int32)
    modes = np.array([sah.EXACT, sah.SAALSH] * 5, np.int32)
    got = ix.rkmips_batch(Q, K, modes=modes)
    for r in range(10):
        exact = oracle.rkmips(W.U, W.P, Q[r], 10)
        if modes[r] == sah.EXACT:
            assert np.array_equal(got[r], exact)
            assert np.array_equal(got[r], ix.rkmips(Q[r], 10))
        else:
            assert set(exact.tolist()) <= set(got[r].tolist())
            assert np.array_equal(got[r], ix.rkmips(Q[r], 10, mode=sah.SAALSH))


def test_fp8_dimension_limit(sah):
    W = workload.make("c1", m=300, n=200, d=128)
    with pytest.raises(sah.SahError) as e:
        sah.Index(W.U, W.P, k_max=10, leaf_size=32, precision=2)
    assert e.value.status == sah.SAH_ERR_UNSUPPORTED
