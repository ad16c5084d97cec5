"""Pins of the FP64 RkMIPS oracle against facts that do not come from the oracle itself.

Def. 1 (RkMIPS) with the tie reading taken from Alg. 2 / Alg. 5: u answers "yes" for
(q, k) iff #{p : <u,p> > <u,q>} < k.  The pins:

* golden: a 2-D example worked by hand (tests/golden/rkmips_2d.json);
* P1 exhaustive enumeration of every score-consistent total order of P u {q} on tiny
  integer inputs (exact scores, frequent ties): u is in the answer iff q sits in the
  first k places of some such order;
* P2 nesting in k; P3 the full user set at k = n (q in P) and k = n + 1 (any q);
* P4 k = 1 against a textbook MIPS (one GEMM plus a row maximum);
* P5 invariances (power-of-two user scaling, user and item permutations, q kept,
  removed or duplicated in P);
* the thresholds tau_u(k) against an independent numpy sort, and the count rule
  against the threshold rule;
* planted mistakes (a non-strict count, a dropped coordinate) fail the pins.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_golden_2d_counts_answers_and_tau():
    g = _load("rkmips_2d.json")
    P = np.array(g["P"], np.float32)
    U = np.array(g["U"], np.float32)
    for case in g["cases"]:
        q = np.array(case["q"], np.float32)
        assert oracle.count_above(U, P, q).tolist() == case["counts"]
        for k, ans in case["answers"].items():
            assert oracle.rkmips(U, P, q, int(k)).tolist() == ans
    t = oracle.tau(U, P, 4)
    assert t[0].tolist() == g["tau"]["u0"]
    assert t[3].tolist() == g["tau"]["u3"]


def _enumeration_answer(P_int, U_int, q_int, q_index_in_P, k):
    """P1: the favourable-tie reading of Def. 1 by brute force over total orders.

    Elements are the items of P, plus q as an extra element when q is not in P.  A total
    order is consistent when scores never increase along it.  u answers "yes" iff q
    appears among the first k elements of at least one consistent order.
    """
    n = len(P_int)
    elems = [tuple(p) for p in P_int]
    qpos = q_index_in_P
    if q_index_in_P is None:
        elems.append(tuple(q_int))
        qpos = n
    out = []
    for ui, u in enumerate(U_int):
        sc = [sum(a * b for a, b in zip(u, e)) for e in elems]   # exact Python integers
        yes = False
        for perm in itertools.permutations(range(len(elems))):
            if all(sc[perm[i]] >= sc[perm[i + 1]] for i in range(len(perm) - 1)):
                if perm.index(qpos) < k:
                    yes = True
                    break
        if yes:
            out.append(ui)
    return out


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("q_in_P", [True, False])
def test_P1_enumeration_tiny_integer(seed, q_in_P):
    n, m, d = 5, 6, 2 + seed % 2
    P, U, q = workload.tie_case(n, m, d, lo=-2, hi=2, seed=seed)
    qi = None
    if q_in_P:
        qi = seed % n
        q = P[qi].copy()
    Pi = P.astype(int).tolist()
    Ui = U.astype(int).tolist()
    qint = q.astype(int).tolist()
    for k in range(1, n + 2):
        expect = _enumeration_answer(Pi, Ui, qint, qi, k)
        assert oracle.rkmips(U, P, q, k).tolist() == expect, (k, q_in_P)


def test_P2_nested_in_k_and_P3_full_set():
    W = workload.make("c1", m=400, n=300)
    for qi in W.query_idx[:4]:
        q = W.P[qi]
        prev = set()
        for k in range(1, 60, 3):
            cur = set(oracle.rkmips(W.U, W.P, q, k).tolist())
            assert prev <= cur
            prev = cur
        assert len(oracle.rkmips(W.U, W.P, q, W.n)) == W.m          # q in P
    foreign = np.random.default_rng(7).standard_normal(W.d).astype(np.float32)
    assert len(oracle.rkmips(W.U, W.P, foreign, W.n + 1)) == W.m


def test_P4_k1_is_textbook_mips():
    W = workload.make("c1", m=500, n=400)
    rng = np.random.default_rng(11)
    q = rng.standard_normal(W.d).astype(np.float32)                     # q not in P
    S = W.U.astype(np.float64) @ W.P.astype(np.float64).T               # one GEMM
    best = S.max(axis=1)                                                # row maximum
    sq = W.U.astype(np.float64) @ q.astype(np.float64)
    scale = np.linalg.norm(W.U, axis=1) * max(np.linalg.norm(W.P, axis=1).max(), np.linalg.norm(q))
    clear = np.abs(sq - best) > 1e-9 * scale
    expect = set(np.flatnonzero((sq >= best) & clear).tolist())
    got = set(oracle.rkmips(W.U, W.P, q, 1).tolist())
    assert got & set(np.flatnonzero(clear).tolist()) == expect
    # exact integer data, q inside P: ties are exact on both sides
    P, U, _ = workload.tie_case(40, 60, 3, lo=-3, hi=3, seed=5)
    q = P[7]
    S = U.astype(np.int64) @ P.astype(np.int64).T
    expect = np.flatnonzero((U.astype(np.int64) @ q.astype(np.int64)) >= S.max(axis=1)).tolist()
    assert oracle.rkmips(U, P, q, 1).tolist() == expect


def test_P5_invariances():
    W = workload.make("c1", m=300, n=250)
    rng = np.random.default_rng(3)
    q = W.P[W.query_idx[0]]
    for k in (1, 5, 10, 40):
        base = oracle.rkmips(W.U, W.P, q, k)
        # power-of-two scaling of users is exact in floating point
        scaled = W.U * np.float32(2.0 ** rng.integers(-6, 7, size=(W.m, 1))).astype(np.float32)
        assert np.array_equal(oracle.rkmips(scaled, W.P, q, k), base)
        # permuting users permutes the ids
        perm = rng.permutation(W.m)
        got = oracle.rkmips(W.U[perm], W.P, q, k)
        assert np.array_equal(np.sort(perm[got]), base)
        # permuting items changes nothing
        assert np.array_equal(oracle.rkmips(W.U, W.P[rng.permutation(W.n)], q, k), base)
        # q kept in P, removed from P, or duplicated: same answer
        qi = W.query_idx[0]
        removed = np.delete(W.P, qi, axis=0)
        dup = np.vstack([W.P, W.P[qi:qi + 1]])
        assert np.array_equal(oracle.rkmips(W.U, removed, q, k), base)
        assert np.array_equal(oracle.rkmips(W.U, dup, q, k), base)


def test_tau_matches_independent_sort_and_count_rule():
    W = workload.make("c2", m=300, n=500)
    kmax = 50
    t = oracle.tau(W.U, W.P, kmax)
    ref = -np.sort(-(W.U.astype(np.float64) @ W.P.astype(np.float64).T), axis=1)[:, :kmax]
    np.testing.assert_allclose(t, ref, rtol=1e-12, atol=1e-12)
    for qi in W.query_idx[:3]:
        q = W.P[qi]
        for k in (1, 5, 10, 20, 50):
            assert np.array_equal(oracle.rkmips(W.U, W.P, q, k), oracle.rkmips_tau(W.U, t, q, k))
    # tau past n is -inf
    t_small = oracle.tau(W.U[:3], W.P[:4], 6)
    assert np.all(np.isneginf(t_small[:, 4:]))


def test_sampled_membership_matches_full_answer():
    W = workload.make("c2", m=800, n=300)
    users = workload.sample_rows(W.m, 100, seed=9)
    q = W.P[W.query_idx[1]]
    full = set(oracle.rkmips(W.U, W.P, q, 10).tolist())
    member = oracle.rkmips_sampled(W.U, W.P, q, 10, users)
    assert [u in full for u in users.tolist()] == member.tolist()


# ------------------------------------------------------------------ planted mistakes
def _mutant_nonstrict(U, P, q, k):
    S = U.astype(np.float64) @ P.astype(np.float64).T
    sq = U.astype(np.float64) @ q.astype(np.float64)
    return np.flatnonzero((S >= sq[:, None]).sum(axis=1) < k).tolist()


def _mutant_dropped_coordinate(U, P, q, k):
    S = U[:, :-1].astype(np.float64) @ P[:, :-1].astype(np.float64).T
    sq = U[:, :-1].astype(np.float64) @ q[:-1].astype(np.float64)
    return np.flatnonzero((S > sq[:, None]).sum(axis=1) < k).tolist()


def test_pins_catch_planted_mistakes():
    g = _load("rkmips_2d.json")
    P = np.array(g["P"], np.float32)
    U = np.array(g["U"], np.float32)
    caught_strict = caught_coord = False
    for case in g["cases"]:
        q = np.array(case["q"], np.float32)
        for k, ans in case["answers"].items():
            caught_strict |= _mutant_nonstrict(U, P, q, int(k)) != ans
            caught_coord |= _mutant_dropped_coordinate(U, P, q, int(k)) != ans
    assert caught_strict and caught_coord
    # P1 also catches the non-strict count on tie-heavy data
    P, U, q = workload.tie_case(5, 6, 2, seed=1)
    q = P[0].copy()
    diffs = 0
    for k in range(1, 6):
        diffs += _mutant_nonstrict(U, P, q, k) != _enumeration_answer(
            P.astype(int).tolist(), U.astype(int).tolist(), q.astype(int).tolist(), 0, k)
    assert diffs > 0


# ------------------------------------------------------------------ margins
def test_golden_margins_and_planted_mistakes():
    """margin_u = |<u,q> - tau_u(k)| / (||u|| ||q||), the distance of a user's decision from
    a tie, against values worked by hand; a wrong k index or a missing norm in the
    denominator changes at least one of them."""
    g = _load("rkmips_2d.json")
    P = np.array(g["P"], np.float32)
    U = np.array(g["U"], np.float32)
    mg = g["margins"]
    q = np.array(mg["q"], np.float32)
    users = np.arange(U.shape[0])
    T = oracle.tau(U, P, 4, users)
    want = {(c["user"], c["k"]): float(c["margin"]) for c in mg["cases"]}
    for (u, k), m in want.items():
        got = oracle.margins(U, T[[u]], q, k, np.array([u]))[0]
        assert got == m if np.isinf(m) else np.isclose(got, m, rtol=1e-15, atol=0.0), (u, k, got, m)

    def mutant(kind, u, k):
        U64, q64 = U.astype(np.float64), q.astype(np.float64)
        sq = U64[u] @ q64
        t = T[u, k if kind == "k_index" else k - 1]
        den = {"no_q_norm": np.linalg.norm(U64[u]), "no_u_norm": np.linalg.norm(q64)}.get(
            kind, np.linalg.norm(U64[u]) * np.linalg.norm(q64))
        return abs(sq - t) / den if den > 0 else np.inf

    for kind in ("k_index", "no_q_norm", "no_u_norm"):
        assert any(not np.isclose(mutant(kind, u, k), m) for (u, k), m in want.items()
                   if np.isfinite(m) and k < 4), kind


def test_margin_scale_invariance_and_zero_at_ties():
    W = workload.make("c2", m=200, n=300)
    users = workload.sample_rows(W.m, 40, seed=4)
    q = W.P[W.query_idx[0]]
    T = oracle.tau(W.U, W.P, 10, users)
    m1 = oracle.margins(W.U, T, q, 10, users)
    T2 = oracle.tau(W.U * 4.0, W.P, 10, users)            # power-of-two scaling is exact
    m2 = oracle.margins(W.U * 4.0, T2, q, 10, users)
    np.testing.assert_allclose(m1, m2, rtol=1e-12)
    # q equal to a user's k-th item: margin 0 for that user at that k
    u = int(users[0])
    s = W.U[u].astype(np.float64) @ W.P.astype(np.float64).T
    kth = int(np.argsort(-s, kind="stable")[2])
    m3 = oracle.margins(W.U, oracle.tau(W.U, W.P, 3, np.array([u])), W.P[kth], 3, np.array([u]))
    assert m3[0] == 0.0
