"""Pins of the step-by-step oracle (oracle/sah.py) against the paper's identities,
lemmas and hand-worked examples, and against the plain-definition oracle."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import sah
import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    with open(os.path.join(GOLDEN, "sah_steps_2d.json")) as f:
        return json.load(f)


def test_golden_sat_eq6_to_eq8():
    g = _golden()["sat"]
    P = np.array(g["P"], float)
    c = P.mean(axis=0)
    R = max(np.linalg.norm(p - c) for p in P)
    assert np.allclose(c, g["c"]) and np.isclose(R, g["R"])
    I0 = sah.sat_item(P[0], c, R)
    Uu = sah.sat_user(np.array(g["u"], float), R)
    # sqrt of a rounding residue of R^2 - ||p - c||^2 is ~1e-8, hence atol
    assert np.allclose(I0, g["I0"], atol=1e-7) and np.allclose(Uu, g["Uu"])
    assert np.isclose(I0 @ Uu / (R * R), g["cos"])


def test_golden_lemma2_lemma3_tight():
    g = _golden()
    l2, l3 = g["lemma2"], g["lemma3"]
    b2 = sah.node_upper_bound(np.array(l2["q"], float), np.array(l2["c"], float), l2["omega"])
    assert np.isclose(b2, l2["bound"])
    assert np.isclose(np.dot(l2["tight_user"], l2["q"]), b2)
    b3 = sah.vector_upper_bound(np.array(l3["q"], float), np.array(l3["c"], float), l3["theta"])
    assert np.isclose(b3, l3["bound"])
    assert np.isclose(np.dot(l3["tight_user"], l3["q"]), b3)


def test_golden_partitions_alg1():
    g = _golden()["partitions"]
    norms = np.array(g["norms"], float)
    P = norms[:, None] * np.eye(1, 3, 0)          # vectors with the given norms
    A = workload.srp_matrix(4, 4).astype(np.float64)
    ix = sah.sa_alsh_index(P, norms, 0, g["b"], A, 1, 4)
    assert [len(s) for s in ix.items] == g["sizes"]
    assert np.allclose(ix.M, g["M"])


def test_golden_cone_tree_alg3():
    g = _golden()["cone_tree"]
    ang = np.deg2rad(g["angles_deg"])
    Uhat = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    for seed in range(8):
        leaves = sah.cone_tree(Uhat, np.arange(len(ang)), g["N0"], seed)
        assert sorted(sorted(l.members.tolist()) for l in leaves) == g["leaves"]


def test_sat_norms_and_eq8_identity_random():
    rng = np.random.default_rng(0)
    P = rng.standard_normal((50, 7)) * rng.lognormal(0, 0.5, (50, 1))
    c = P.mean(axis=0)
    R = max(np.linalg.norm(p - c) for p in P)
    for _ in range(20):
        u = rng.standard_normal(7)
        Uu = sah.sat_user(u, R)
        assert np.isclose(np.linalg.norm(Uu), R)
        for p in P[:10]:
            I = sah.sat_item(p, c, R)
            assert np.isclose(np.linalg.norm(I), R)
            assert np.isclose(I @ Uu / (R * R), (p - c) @ u / (R * np.linalg.norm(u)))
        # Fact 1: the shift does not move the argmax over items
        scores_sat = [sah.sat_item(p, c, R) @ Uu for p in P]
        assert int(np.argmax(scores_sat)) == int(np.argmax(P @ u))


def test_srp_collision_probability_eq2():
    rng = np.random.default_rng(1)
    d, N = 16, 10000
    A = rng.standard_normal((N, d))
    for target in (0.3, 1.0, 2.0, 2.8):
        x = rng.standard_normal(d)
        x /= np.linalg.norm(x)
        y0 = rng.standard_normal(d)
        y0 -= (y0 @ x) * x
        y0 /= np.linalg.norm(y0)
        y = np.cos(target) * x + np.sin(target) * y0
        delta = sah.angle(x, y)
        hit = np.mean(sah.srp_bits(A, x) == sah.srp_bits(A, y))
        p = 1 - delta / np.pi
        assert abs(hit - p) < 4 * np.sqrt(p * (1 - p) / N) + 1e-9


def _random_cone(rng, d, m, omega):
    c = rng.standard_normal(d)
    c /= np.linalg.norm(c)
    out = []
    while len(out) < m:
        v = rng.standard_normal(d)
        v /= np.linalg.norm(v)
        if sah.angle(v, c) <= omega:
            out.append(v)
        else:  # pull towards the centre until inside
            t = rng.uniform(0, 1)
            w = t * c + (1 - t) * v
            w /= np.linalg.norm(w)
            if sah.angle(w, c) <= omega:
                out.append(w)
    return c, np.array(out)


def test_lemma2_lemma3_hold_on_random_cones():
    rng = np.random.default_rng(2)
    for trial in range(40):
        d = 3 + trial % 6
        omega = rng.uniform(0.1, 2.5)
        c, X = _random_cone(rng, d, 30, omega)
        mean = X.mean(axis=0)
        om = max(sah.angle(x, mean) for x in X)
        for _ in range(5):
            q = rng.standard_normal(d) * rng.lognormal()
            nb = sah.node_upper_bound(q, mean, om)
            assert (X @ q).max() <= nb + 1e-12
            for x in X[:8]:
                vb = sah.vector_upper_bound(q, mean, sah.angle(x, mean))
                assert x @ q <= vb + 1e-12
                assert vb <= np.linalg.norm(q) + 1e-12       # never looser than Cauchy-Schwarz


def test_cone_tree_invariants_alg3():
    W = workload.make("c2", m=3000, n=10)
    U = W.U.astype(np.float64)
    Uhat = U / np.linalg.norm(U, axis=1, keepdims=True)
    leaves = sah.cone_tree(Uhat, np.arange(W.m), 20, seed=5)
    allm = np.concatenate([l.members for l in leaves])
    assert np.array_equal(np.sort(allm), np.arange(W.m))          # disjoint cover
    for l in leaves:
        assert 1 <= len(l.members) <= 20
        assert np.allclose(l.center, Uhat[l.members].mean(axis=0))
        assert np.all(l.theta <= l.omega + 1e-12)


def test_alg1_partition_invariants():
    W = workload.make("c2", m=10, n=2000)
    P = W.P.astype(np.float64)
    nrm = np.linalg.norm(P, axis=1)
    order = np.argsort(-nrm, kind="stable")
    A = workload.srp_matrix(16, W.d + 1).astype(np.float64)
    ix = sah.sa_alsh_index(P[order], nrm[order], 200, 0.5, A, 4, 4)
    cover = np.concatenate(ix.items)
    assert np.array_equal(cover, np.arange(200, 2000))
    assert np.all(np.diff(ix.M) < 0)
    for S, M in zip(ix.items, ix.M):
        assert np.all(nrm[order][S] <= M) and np.all(nrm[order][S] > 0.5 * M)


def test_alg4_bound_chain():
    W = workload.make("c2", m=600, n=800)
    ix = sah.sah_index(W.P, W.U, kmax=20, N0=20, p_prime=60)
    Uhat = ix.Uhat
    T = oracle.tau(Uhat.astype(np.float32), W.P, 20)     # tau of the unit users (fp32 inputs)
    for bi, blk in enumerate(ix.blocks):
        assert np.all(ix.LB[bi] <= ix.L[blk.members] + 1e-12)
    assert np.all(ix.L <= T + 1e-6)                               # P' scores <= tau over P
    assert np.all(ix.norms[:20][None, :] >= T - 1e-6)             # ||p_k|| >= tau(k), unit u


def test_alg5_exact_mode_equals_definition():
    W = workload.make("c2", m=700, n=900)
    for p_prime in (20, 80, 900):
        ix = sah.sah_index(W.P, W.U, kmax=20, N0=20, p_prime=p_prime, seed=3)
        for qi in W.query_idx[:3]:
            q = W.P[qi]
            for k in (1, 5, 20, 25):
                got = sah.sah_query(ix, q, k, "exact")
                ref = oracle.rkmips(W.U, W.P, q, k)
                assert np.array_equal(got, ref), (p_prime, k)


def test_alg5_saalsh_mode_superset_and_full_probe_is_exact():
    W = workload.make("c2", m=300, n=600)
    code_bits, n_tables = 4, 3
    A = workload.srp_matrix(n_tables * code_bits, W.d + 1, seed=4).astype(np.float64)
    ix = sah.sah_index(W.P, W.U, kmax=10, N0=20, p_prime=40, A=A, n_tables=n_tables,
                       code_bits=code_bits, seed=1)
    for qi in W.query_idx[:3]:
        q = W.P[qi]
        for k in (1, 10):
            exact = set(oracle.rkmips(W.U, W.P, q, k).tolist())
            approx = set(sah.sah_query(ix, q, k, "saalsh", probe_radius=0).tolist())
            assert exact <= approx                                   # every "no" is sound
            full = set(sah.sah_query(ix, q, k, "saalsh", probe_radius=code_bits).tolist())
            assert full == exact


def test_zero_norm_users_always_answer_yes():
    W = workload.make("c1", m=50, n=60)
    U = W.U.copy()
    U[[3, 17]] = 0.0
    ix = sah.sah_index(W.P, U, kmax=10, N0=8, p_prime=20)
    got = sah.sah_query(ix, W.P[W.query_idx[0]], 1)
    assert {3, 17} <= set(got.tolist())
    assert {3, 17} <= set(oracle.rkmips(U, W.P, W.P[W.query_idx[0]], 1).tolist())


def test_splitmix64_reference_values():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 0: the first output of the
    # generator whose state starts at 0 is 0xE220A8397B1DCDAF.
    assert sah.splitmix64(0) == 0xE220A8397B1DCDAF
    # second output: state advanced by the golden gamma once more
    assert sah.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


# ------------------------------------------------------------------ SimHash candidate rule
def _simhash_golden():
    with open(os.path.join(GOLDEN, "simhash_2x3.json")) as f:
        return json.load(f)


def _simhash_state(g):
    P = np.array(g["P"], float)
    norms = np.linalg.norm(P, axis=1)
    A = np.array(g["A"], float)
    ix = sah.sa_alsh_index(P, norms, 0, g["b"], A, g["n_tables"], g["code_bits"])
    uc = sah.user_codes(ix, np.array(g["u"], float), float(ix.radii[0]))
    cands = {r: sorted(sah.simhash_candidates(ix, 0, uc, int(r))) for r in g["candidates"]}
    return P, ix, uc, cands


def _simhash_matches(g, state):
    P, ix, uc, cands = state
    return (len(ix.items) == 1 and ix.codes[0].tolist() == g["item_codes"]
            and uc.tolist() == g["user_codes"]
            and all(cands[r] == g["candidates"][r] for r in g["candidates"]))


def test_golden_simhash_codes_and_candidates():
    """Eq. 1, Eq. 9 and Alg. 1's K tables of code_bits SRP bits, against a case worked by
    hand: the partition, its centroid and radius, every item's and the user's code per
    table, and the candidate set at probe radius 0, 1, 2 and 3."""
    g = _simhash_golden()
    P, ix, uc, cands = state = _simhash_state(g)
    assert [len(s) for s in ix.items] == [6]
    assert np.allclose(ix.centroids[0], g["centroid"]) and np.isclose(ix.radii[0], g["R"])
    assert ix.codes[0].tolist() == g["item_codes"]
    assert uc.tolist() == g["user_codes"]
    for r, want in g["candidates"].items():
        assert cands[r] == want, r
    assert _simhash_matches(g, state)
    # buckets: each table maps a code to the items that carry it
    for t in range(g["n_tables"]):
        for code, members in ix.tables[0][t].items():
            assert all(g["item_codes"][i][t] == code for i in members)


def test_golden_alg2_decisions_by_probe_radius():
    """Alg. 2 on the hand-worked index: a radius-0 probe misses an item that beats <u,q>
    and answers "yes" where the definition says "no"; radius 1 finds it."""
    g = _simhash_golden()
    P, ix, _, _ = _simhash_state(g)
    u = np.array(g["u"], float)
    a2 = g["alg2"]
    q = P[a2["q_item"]]
    assert int(np.count_nonzero(P @ u > q @ u)) == a2["exact_count_above"]
    for c in a2["cases"]:
        got = sah.sa_alsh_decide(ix, P, u, q, c["k"], np.array([], dtype=int), c["probe_radius"])
        assert got == c["yes"], c


def test_simhash_pins_catch_planted_mistakes(monkeypatch):
    """Each plausible slip in the candidate rule fails the golden case: a strict Hamming
    test, bits assigned to tables column-wise instead of row-wise, sgn(0) read as -1, and
    the bits of a code packed in reverse order."""
    g = _simhash_golden()
    orig_pack, orig_bits, orig_cand = sah.pack_codes, sah.sign_bits, sah.simhash_candidates

    def strict_candidates(index, j, ucodes, probe_radius):
        out = set()
        for t in range(index.n_tables):
            for code, members in index.tables[j][t].items():
                if bin(code ^ int(ucodes[t])).count("1") < probe_radius:
                    out.update(members)
        return out

    def transposed_pack(bits, n_tables, code_bits):
        bits = np.atleast_2d(bits).astype(np.uint64)
        out = np.zeros((bits.shape[0], n_tables), dtype=np.uint64)
        for t in range(n_tables):
            for b in range(code_bits):
                out[:, t] |= bits[:, b * n_tables + t] << np.uint64(b)
        return out

    def reversed_pack(bits, n_tables, code_bits):
        bits = np.atleast_2d(bits).astype(np.uint64)
        out = np.zeros((bits.shape[0], n_tables), dtype=np.uint64)
        for t in range(n_tables):
            for b in range(code_bits):
                out[:, t] |= bits[:, t * code_bits + b] << np.uint64(code_bits - 1 - b)
        return out

    def negative_zero_bits(proj):
        return (np.asarray(proj, np.float64) > 0.0).astype(np.uint8)

    caught = {}
    with monkeypatch.context() as mp:
        mp.setattr(sah, "simhash_candidates", strict_candidates)
        caught["strict_hamming"] = not _simhash_matches(g, _simhash_state(g))
    with monkeypatch.context() as mp:
        mp.setattr(sah, "pack_codes", transposed_pack)
        caught["table_bit_mixup"] = not _simhash_matches(g, _simhash_state(g))
    with monkeypatch.context() as mp:
        mp.setattr(sah, "pack_codes", reversed_pack)
        caught["reversed_bits"] = not _simhash_matches(g, _simhash_state(g))
    with monkeypatch.context() as mp:
        mp.setattr(sah, "sign_bits", negative_zero_bits)
        caught["sgn0_minus"] = not _simhash_matches(g, _simhash_state(g))
    assert sah.pack_codes is orig_pack and sah.sign_bits is orig_bits and sah.simhash_candidates is orig_cand
    assert all(caught.values()), caught


# ------------------------------------------------------------------ QNF (H2-ALSH) and kMIPS
def _qnf_golden():
    with open(os.path.join(GOLDEN, "qnf_sat_3items.json")) as f:
        return json.load(f)


def _qnf_index(g, transform):
    P = np.array(g["P"], float)
    order = np.array(g["order"])
    Ps = P[order]
    A = np.array(g["A"], float)
    ix = sah.sa_alsh_index(Ps, np.linalg.norm(Ps, axis=1), 0, g["b"], A, g["n_tables"], g["code_bits"],
                           transform)
    return P, order, Ps, ix


def test_golden_qnf_and_sat_codes():
    """Eq. 3-4 against Eq. 6-7 on a case worked by hand: QNF keeps the items unshifted
    and pads them to norm M, SAT shifts them by the centroid and pads to R; one item's
    codes differ between the two, and the user's codes do not."""
    g = _qnf_golden()
    for tr in ("sat", "qnf"):
        P, order, Ps, ix = _qnf_index(g, tr)
        assert [len(s) for s in ix.items] == [3]
        assert np.allclose(ix.centroids[0], g[tr]["centroid"]) and np.isclose(ix.radii[0] ** 2, g[tr]["R2"])
        by_item = np.empty((3, 2), dtype=np.int64)
        by_item[order] = ix.codes[0].astype(np.int64)
        assert by_item.tolist() == g[tr]["codes_by_item"], tr
        uc = sah.user_codes(ix, np.array(g["u"], float), float(ix.radii[0]))
        assert uc.tolist() == g["user_codes"]
    # Eq. 5: ||I(p) - U(u)||^2 = 2 M (M - <p, u> / ||u||) under QNF
    M = np.sqrt(20.0)
    u = np.array(g["u"], float)
    for p in np.array(g["P"], float):
        lhs = np.sum((sah.qnf_item(p, M) - sah.qnf_user(u, M)) ** 2)
        assert np.isclose(lhs, 2 * M * (M - p @ u / np.linalg.norm(u)))


def test_golden_kmips_by_transform_and_radius():
    g = _qnf_golden()
    u = np.array(g["u"], float)
    for c in g["kmips"]:
        P, order, Ps, ix = _qnf_index(g, c["transform"])
        pos = sah.sa_alsh_kmips(ix, Ps, u, c["k"], np.array([], dtype=int), c["probe_radius"])
        assert order[pos].tolist() == c["items"], c


def test_qnf_pins_catch_a_shifted_qnf():
    """A QNF that shifts by the centroid (SAT's step) gives SAT's codes, which the golden
    QNF codes reject."""
    g = _qnf_golden()
    P, order, Ps, ix_sat = _qnf_index(g, "sat")
    by_item = np.empty((3, 2), dtype=np.int64)
    by_item[order] = ix_sat.codes[0].astype(np.int64)
    assert by_item.tolist() != g["qnf"]["codes_by_item"]


@pytest.mark.parametrize("transform", ["sat", "qnf"])
def test_kmips_full_probe_is_exact_topk(transform):
    """With the probe radius at code_bits every item of a visited partition is a candidate,
    and the mu_j stop only skips partitions that cannot beat phi: the answer is the exact
    top-k (brute force in FP64)."""
    W = workload.make("c1", n=300, m=20, d=8)
    norms = np.linalg.norm(W.P.astype(np.float64), axis=1)
    order = np.argsort(-norms, kind="stable")
    Ps = W.P.astype(np.float64)[order]
    rng = np.random.default_rng(5)
    A = rng.standard_normal((6 * 4, 9))
    ix = sah.sa_alsh_index(Ps, norms[order], 10, 0.5, A, 6, 4, transform)
    for i in range(8):
        u = W.U[i].astype(np.float64)
        for k in (1, 5, 20):
            got = sah.sa_alsh_kmips(ix, Ps, u, k, np.arange(10), 4)
            sc = Ps @ u
            want = np.lexsort((np.arange(len(sc)), -sc))[:k]
            assert np.array_equal(got, want), (transform, i, k)


def test_kmips_answer_is_best_of_candidates():
    """At radius 0 the answer is the k best of the seed and the collected candidates, in
    descending score, and every answer item beats or ties every other candidate."""
    W = workload.make("c1", n=400, m=10, d=8)
    norms = np.linalg.norm(W.P.astype(np.float64), axis=1)
    order = np.argsort(-norms, kind="stable")
    Ps = W.P.astype(np.float64)[order]
    A = np.random.default_rng(6).standard_normal((8 * 3, 9))
    ix = sah.sa_alsh_index(Ps, norms[order], 5, 0.5, A, 8, 3)
    for i in range(10):
        u = W.U[i].astype(np.float64)
        got = sah.sa_alsh_kmips(ix, Ps, u, 10, np.arange(5), 0)
        sc = Ps[got] @ u
        assert np.all(np.diff(sc) <= 0)
        assert len(got) == 10                     # the seed alone holds 5; candidates add the rest
        # the seed is always in C: a seed item left out cannot beat the answer's last
        for i in set(range(5)) - set(got.tolist()):
            assert Ps[i] @ u <= sc[-1]
