"""SAH's algorithms restated step by step in numpy FP64, for small inputs.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Each function follows one
passage of the paper, in the paper's order and notation:

* SRP hashing ................ Eq. 1 (h_srp(p) = sgn(<a, p>)), collision rate Eq. 2
* QNF (H2-ALSH) .............. Eq. 3 (item transform), Eq. 4 (user transform), Eq. 5
* SAT ........................ Eq. 6 (item transform), Eq. 7 (user transform), Eq. 8
* SA-ALSH family ............. Eq. 9
* SA-ALSH indexing ........... Alg. 1
* SA-ALSH query .............. Alg. 2
* Node / vector upper bounds . Lemma 2 (Eq. 11), Lemma 3 (Eq. 12)
* Cone-Tree construction ..... Alg. 3
* SAH indexing ............... Alg. 4
* SAH query .................. Alg. 5

Readings where the paper is silent (each is also listed with the design notes):
* Ties: the count rule, u answers "yes" iff #{p : <u,p> > <u,q>} < k.
* |P'| = "O(k_max)" is a parameter ``p_prime``.
* SA-ALSH is built on P \\ P' (Alg. 4) while Alg. 2's phi ranges over the candidates C
  only; C is seeded with P', so phi starts at L_u^k and stays a lower bound of the
  true k-th largest score.  The seeded C is checked against <u,q> before the loop.
* A SimHash table is a concatenation of ``code_bits`` SRP bits; ``n_tables`` tables;
  one projection matrix shared by all partitions; a candidate is an item whose code is
  within Hamming distance ``probe_radius`` of the user's code in at least one table;
  sgn(0) := +1.
* Users enter the bounds as unit vectors (Fact 2).  Zero-norm users score 0 against
  every item, so they always answer "yes" and stay out of the Cone-Tree.
* A node whose centre is the zero vector gets omega = pi.  A split that leaves one side
  empty (all users collinear) splits the node's list into halves.
* Alg. 3's random point v: position splitmix64(splitmix64(seed) ^ key) mod |N| in the
  node's list, where the root's key is 1 and the children of key x have keys 2x and
  2x + 1 (mod 2^64).  SplitMix64 is Steele, Lea and Flood's generator (OOPSLA 2014).
* Alg. 1 with a partition maximum M_j = 0 would never end: all zero-norm items form one
  final partition.
* QNF in place of SAT (the paper's H2-ALSH comparison): the same norm partitions and
  SimHash tables, each partition transformed by Eq. 3 with M = M_j, its largest norm
  (H2-ALSH's homocentric partitions), and users by Eq. 4.
* Standalone kMIPS (the paper's SA-ALSH vs H2-ALSH comparison): Alg. 2's candidate loop
  without a query item: C seeded with P', partitions in order, stop once the k-th largest
  score phi of C exceeds mu_j = M_j ||u||; the answer is the k best of C.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

import numpy as np

MASK64 = (1 << 64) - 1


def ips(X: np.ndarray, v: np.ndarray) -> np.ndarray:
    """<x, v> for every row x of X, in FP64.  One reduction per row, so identical rows
    (q and its own copy inside P) always give identical scores."""
    X = np.atleast_2d(np.asarray(X, np.float64))
    return (X * np.asarray(v, np.float64)[None, :]).sum(axis=1)


# ----------------------------------------------------------------------------- RNG
def splitmix64(x: int) -> int:
    """SplitMix64 output function applied to state x + golden gamma (one step)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def pivot_position(seed: int, key: int, size: int) -> int:
    """Index of Alg. 3's random point v inside a node's member list."""
    return splitmix64(splitmix64(seed & MASK64) ^ (key & MASK64)) % size


# ----------------------------------------------------------------------------- SRP / SAT
def sign_bits(proj: np.ndarray) -> np.ndarray:
    """Eq. 1's sign as a bit: 1 where sgn(projection) = +1, with sgn(0) := +1."""
    return (np.asarray(proj, np.float64) >= 0.0).astype(np.uint8)


def srp_bits(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Eq. 1 for every row of A: bit 1 where sgn(<a, x>) = +1 (sgn(0) := +1)."""
    return sign_bits(np.asarray(A, np.float64) @ np.asarray(x, np.float64))


def srp_projections(A: np.ndarray, X: np.ndarray) -> np.ndarray:
    """<a, x> for every projection row a and every row x (rows x projections)."""
    return np.asarray(X, np.float64) @ np.asarray(A, np.float64).T


def pack_codes(bits: np.ndarray, n_tables: int, code_bits: int) -> np.ndarray:
    """Table t's code = sum_b bit[t*code_bits + b] << b (one row per vector)."""
    bits = np.atleast_2d(bits).astype(np.uint64)
    out = np.zeros((bits.shape[0], n_tables), dtype=np.uint64)
    for t in range(n_tables):
        for b in range(code_bits):
            out[:, t] |= bits[:, t * code_bits + b] << np.uint64(b)
    return out


def sat_item(p: np.ndarray, c: np.ndarray, R: float) -> np.ndarray:
    """Eq. 6: I(p, c) = [p - c; sqrt(R^2 - ||p - c||^2)] (radicand clamped at 0)."""
    diff = np.asarray(p, np.float64) - np.asarray(c, np.float64)
    rad = R * R - float(diff @ diff)
    return np.concatenate([diff, [np.sqrt(max(rad, 0.0))]])


def qnf_item(p: np.ndarray, M: float) -> np.ndarray:
    """Eq. 3: I(p) = [p; sqrt(M^2 - ||p||^2)] (radicand clamped at 0)."""
    p = np.asarray(p, np.float64)
    rad = M * M - float(p @ p)
    return np.concatenate([p, [np.sqrt(max(rad, 0.0))]])


def qnf_user(u: np.ndarray, M: float) -> np.ndarray:
    """Eq. 4: U(u) = [lambda u; 0] with lambda = M / ||u||."""
    u = np.asarray(u, np.float64)
    nu = np.sqrt(u @ u)
    lam = M / nu if nu > 0 else 0.0
    return np.concatenate([lam * u, [0.0]])


def sat_user(u: np.ndarray, R: float) -> np.ndarray:
    """Eq. 7: U(u) = [lambda u; 0] with lambda = R / ||u||."""
    u = np.asarray(u, np.float64)
    nu = np.sqrt(u @ u)
    lam = R / nu if nu > 0 else 0.0
    return np.concatenate([lam * u, [0.0]])


# ----------------------------------------------------------------------------- SA-ALSH
@dataclasses.dataclass
class SAALSHIndex:
    items: List[np.ndarray]                # per partition: item ids (positions in sorted P)
    M: np.ndarray                          # per partition: max norm M_j
    centroids: List[np.ndarray]            # c_j
    radii: np.ndarray                      # R_j
    codes: List[np.ndarray]                # per partition: |S_j| x n_tables item codes
    tables: List[List[Dict[int, List[int]]]]  # per partition, per table: code -> item ids
    n_tables: int
    code_bits: int
    A: np.ndarray                          # (n_tables*code_bits) x (d+1) projections
    transform: str = "sat"                 # "sat" (Eq. 6, 7) or "qnf" (Eq. 3, 4)


def sa_alsh_index(P_sorted: np.ndarray, norms_sorted: np.ndarray, first: int, b: float,
                  A: np.ndarray, n_tables: int, code_bits: int, transform: str = "sat") -> SAALSHIndex:
    """Alg. 1 on the items at positions first..n-1 of the descending-norm order.

    Partition S_j starts at the largest remaining norm M_j and takes every following
    item with ||p|| > b * M_j; zero-norm items form one final partition.  Per partition:
    centroid c_j, radius R_j = max ||p - c_j||, the SAT item transform of every member,
    and ``n_tables`` SimHash tables keyed by the packed SRP code.  With transform "qnf"
    every member gets Eq. 3's transform with M = M_j instead (no shift: c_j = 0, R_j = M_j).
    """
    assert transform in ("sat", "qnf")
    n = P_sorted.shape[0]
    parts, Ms = [], []
    i = first
    while i < n:
        Mj = float(norms_sorted[i])
        j0 = i
        if Mj == 0.0:
            i = n
        else:
            while i < n and norms_sorted[i] > b * Mj:
                i += 1
        parts.append(np.arange(j0, i))
        Ms.append(Mj)
    cents, radii, codes, tables = [], [], [], []
    for S, Mj in zip(parts, Ms):
        X = np.asarray(P_sorted[S], np.float64)
        if transform == "qnf":
            c = np.zeros(X.shape[1])
            R = float(Mj)
            I = np.stack([qnf_item(x, R) for x in X])
        else:
            c = X.mean(axis=0)
            R = float(np.max(np.sqrt(((X - c) ** 2).sum(axis=1))))
            I = np.stack([sat_item(x, c, R) for x in X])
        bits = sign_bits(srp_projections(A, I))
        cd = pack_codes(bits, n_tables, code_bits)
        tab = []
        for t in range(n_tables):
            buckets: Dict[int, List[int]] = {}
            for row, item in enumerate(S):
                buckets.setdefault(int(cd[row, t]), []).append(int(item))
            tab.append(buckets)
        cents.append(c)
        radii.append(R)
        codes.append(cd)
        tables.append(tab)
    return SAALSHIndex(items=parts, M=np.asarray(Ms), centroids=cents, radii=np.asarray(radii),
                       codes=codes, tables=tables, n_tables=n_tables, code_bits=code_bits,
                       A=np.asarray(A, np.float64), transform=transform)


def user_codes(index: SAALSHIndex, u: np.ndarray, R: float) -> np.ndarray:
    """Eq. 9 for a user: SRP codes of U(u) (Eq. 7; Eq. 4 under QNF) in every table."""
    x = qnf_user(u, R) if index.transform == "qnf" else sat_user(u, R)
    bits = srp_bits(index.A, x)
    return pack_codes(bits, index.n_tables, index.code_bits)[0]


def simhash_candidates(index: SAALSHIndex, j: int, ucodes: np.ndarray,
                       probe_radius: int) -> set:
    """Items of S_j whose code is within Hamming ``probe_radius`` of u's in some table."""
    out = set()
    for t in range(index.n_tables):
        cu = int(ucodes[t])
        for code, members in index.tables[j][t].items():
            if bin(code ^ cu).count("1") <= probe_radius:
                out.update(members)
    return out


def kth_largest(values: np.ndarray, k: int) -> float:
    if len(values) < k:
        return -np.inf
    return float(np.sort(values)[::-1][k - 1])


def sa_alsh_decide(index: SAALSHIndex, P_sorted: np.ndarray, u: np.ndarray, q: np.ndarray,
                   k: int, seed_items: np.ndarray, probe_radius: int,
                   trace: Optional[list] = None) -> bool:
    """Alg. 2: does q stay in u's kMIPS answer?  C starts as ``seed_items`` (P').

    ``trace`` (optional) receives every comparison the decision makes, in order, as
    ("phi", <u,q>, phi) and ("mu", phi, mu_j); it changes nothing in the decision."""
    u = np.asarray(u, np.float64)
    P64 = np.asarray(P_sorted, np.float64)
    sq = float(ips(np.asarray(q, np.float64), u)[0])
    nu = float(np.sqrt(u @ u))
    C = set(int(i) for i in seed_items)
    phi = kth_largest(ips(P64[sorted(C)], u), k) if C else -np.inf
    if trace is not None:
        trace.append(("phi", sq, phi))
    if sq < phi:
        return False
    for j in range(len(index.items)):
        mu = index.M[j] * nu
        if trace is not None:
            trace.append(("mu", phi, mu))
        if phi > mu:
            return True
        ucodes = user_codes(index, u, float(index.radii[j]))
        C |= simhash_candidates(index, j, ucodes, probe_radius)
        phi = kth_largest(ips(P64[sorted(C)], u), k)
        if trace is not None:
            trace.append(("phi", sq, phi))
        if sq < phi:
            return False
    return True


def sa_alsh_kmips(index: SAALSHIndex, P_sorted: np.ndarray, u: np.ndarray, k: int,
                  seed_items: np.ndarray, probe_radius: int) -> np.ndarray:
    """kMIPS of u by the candidate loop of Alg. 2 (no query item): C starts as
    ``seed_items``; partition by partition, stop once phi, the k-th largest score in C,
    exceeds mu_j = M_j ||u||, else add S_j's SimHash candidates.  Returns the positions
    (in P_sorted) of C's k largest scores, best first (equal scores: lower position
    first); fewer than k when C holds fewer."""
    u = np.asarray(u, np.float64)
    P64 = np.asarray(P_sorted, np.float64)
    nu = float(np.sqrt(u @ u))
    C = set(int(i) for i in seed_items)
    phi = kth_largest(ips(P64[sorted(C)], u), k) if C else -np.inf
    for j in range(len(index.items)):
        if phi > index.M[j] * nu:
            break
        ucodes = user_codes(index, u, float(index.radii[j]))
        C |= simhash_candidates(index, j, ucodes, probe_radius)
        phi = kth_largest(ips(P64[sorted(C)], u), k) if C else -np.inf
    pos = np.asarray(sorted(C), dtype=np.int64)
    if len(pos) == 0:
        return pos
    sc = ips(P64[pos], u)
    order = np.lexsort((pos, -sc))
    return pos[order][:k]


# ----------------------------------------------------------------------------- Cone-Tree
def node_upper_bound(q: np.ndarray, c: np.ndarray, omega: float) -> float:
    """Lemma 2 (Eq. 11): ||q|| cos({phi - omega}_+), phi = angle(q, c)."""
    phi = angle(q, c)
    return float(np.linalg.norm(q) * np.cos(max(phi - omega, 0.0)))


def vector_upper_bound(q: np.ndarray, c: np.ndarray, theta_u: float) -> float:
    """Lemma 3 (Eq. 12): ||q|| cos(|phi - theta_u|), phi = angle(q, c)."""
    phi = angle(q, c)
    return float(np.linalg.norm(q) * np.cos(abs(phi - theta_u)))


def angle(x: np.ndarray, y: np.ndarray) -> float:
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    den = np.sqrt(x @ x) * np.sqrt(y @ y)
    if den == 0.0:
        return float(np.pi / 2)
    return float(np.arccos(np.clip((x @ y) / den, -1.0, 1.0)))


@dataclasses.dataclass
class Leaf:
    members: np.ndarray   # user ids, in the node's list order
    center: np.ndarray    # N.c (mean of the unit user vectors)
    omega: float          # N.omega
    theta: np.ndarray     # theta_u per member
    key: int


def cone_tree(Uhat: np.ndarray, ids: np.ndarray, N0: int, seed: int, key: int = 1) -> List[Leaf]:
    """Alg. 3 on the unit vectors Uhat[ids]; returns the leaves, left subtree first."""
    X = np.asarray(Uhat[ids], np.float64)
    c = X.mean(axis=0)
    nc = np.sqrt(c @ c)
    if nc > 0:
        cosang = np.clip((X @ c) / (np.sqrt((X * X).sum(axis=1)) * nc), -1.0, 1.0)
        ang = np.arccos(cosang)
        omega = float(ang.max())
    else:
        ang = np.full(len(ids), np.pi / 2)
        omega = float(np.pi)
    if len(ids) > N0:
        v = X[pivot_position(seed, key, len(ids))]
        l = int(np.argmin(X @ v))            # argmin returns the first minimum
        ul = X[l]
        r = int(np.argmin(X @ ul))
        ur = X[r]
        left_mask = (X @ ul) >= (X @ ur)
        if left_mask.all() or not left_mask.any():
            half = len(ids) // 2
            left_mask = np.zeros(len(ids), dtype=bool)
            left_mask[:half] = True
        kl = (2 * key) & MASK64
        kr = (2 * key + 1) & MASK64
        return (cone_tree(Uhat, ids[left_mask], N0, seed, kl)
                + cone_tree(Uhat, ids[~left_mask], N0, seed, kr))
    return [Leaf(members=np.asarray(ids), center=c, omega=omega, theta=ang, key=key)]


# ----------------------------------------------------------------------------- SAH
@dataclasses.dataclass
class SAHIndex:
    P_sorted: np.ndarray      # items in descending norm order (FP64)
    order: np.ndarray         # P_sorted[i] = P[order[i]]
    norms: np.ndarray         # descending item norms
    p_prime: int
    kmax: int
    L: np.ndarray             # m x kmax lower bounds for unit users (-inf where undefined)
    blocks: List[Leaf]
    LB: np.ndarray            # n_blocks x kmax block lower bounds
    Uhat: np.ndarray
    zero_users: np.ndarray
    saalsh: Optional[SAALSHIndex]


def sah_index(P, U, kmax: int = 50, N0: int = 20, p_prime: Optional[int] = None, b: float = 0.5,
              A: Optional[np.ndarray] = None, n_tables: int = 8, code_bits: int = 4,
              seed: int = 0, transform: str = "sat") -> SAHIndex:
    """Alg. 4: item norms and descending sort, P' lower bounds, SA-ALSH on P \\ P',
    Cone-Tree over the users, and the per-block lower-bound arrays."""
    P = np.asarray(P, np.float64)
    U = np.asarray(U, np.float64)
    n = P.shape[0]
    norms = np.sqrt((P * P).sum(axis=1))
    order = np.argsort(-norms, kind="stable")
    Ps, ns = P[order], norms[order]
    pp = min(n, 4 * kmax if p_prime is None else int(p_prime))
    unorm = np.sqrt((U * U).sum(axis=1))
    zero = np.flatnonzero(unorm == 0.0)
    nz = np.flatnonzero(unorm > 0.0)
    Uhat = np.zeros_like(U)
    Uhat[nz] = U[nz] / unorm[nz, None]
    L = np.full((U.shape[0], kmax), -np.inf)
    if pp > 0:
        for i in range(U.shape[0]):               # kmax-MIPS of every unit user on P'
            top = -np.sort(-ips(Ps[:pp], Uhat[i]))[:kmax]
            L[i, :top.shape[0]] = top
    sa = None
    if A is not None:
        sa = sa_alsh_index(Ps, ns, pp, b, A, n_tables, code_bits, transform)
    blocks = cone_tree(Uhat, nz, N0, seed) if len(nz) else []
    LB = np.array([L[blk.members].min(axis=0) for blk in blocks]).reshape(len(blocks), kmax)
    return SAHIndex(P_sorted=Ps, order=order, norms=ns, p_prime=pp, kmax=kmax, L=L,
                    blocks=blocks, LB=LB, Uhat=Uhat, zero_users=zero, saalsh=sa)


def sah_query(ix: SAHIndex, q, k: int, mode: str = "exact", probe_radius: int = 0,
              trace: Optional[Dict[int, list]] = None) -> np.ndarray:
    """Alg. 5: block test (Lemma 2), user test (Lemma 3), <u,q> vs L_i^k, ||p_k|| test, and
    the kMIPS decision (``exact``: the count rule; ``saalsh``: Alg. 2).  Ascending ids.

    ``trace`` (optional) receives, per user that reaches the <u,q> tests, every comparison
    its decision makes: ("L", <u,q>, L_u^k), ("pk", <u,q>, ||p_k||), then those of
    ``sa_alsh_decide``; it changes no decision."""
    q = np.asarray(q, np.float64)
    n = ix.P_sorted.shape[0]
    nq = float(np.sqrt(q @ q))
    pk = ix.norms[k - 1] if k <= n else -np.inf
    out = list(ix.zero_users.tolist())
    for bi, blk in enumerate(ix.blocks):
        LBk = ix.LB[bi, k - 1] if k <= ix.kmax else -np.inf
        phi = angle(q, blk.center)
        if nq * np.cos(max(phi - blk.omega, 0.0)) < LBk:
            continue
        for u, th in zip(blk.members, blk.theta):
            Lk = ix.L[u, k - 1] if k <= ix.kmax else -np.inf
            if nq * np.cos(abs(phi - th)) < Lk:
                continue
            uh = ix.Uhat[u]
            s = float(ips(q, uh)[0])
            tr = None
            if trace is not None:
                tr = trace.setdefault(int(u), [])
                tr.append(("L", s, Lk))
                tr.append(("pk", s, pk))
            if s < Lk:
                continue
            if pk > s:
                if mode == "exact":
                    yes = int(np.count_nonzero(ips(ix.P_sorted, uh) > s)) < k
                else:
                    yes = sa_alsh_decide(ix.saalsh, ix.P_sorted, uh, q, k,
                                         np.arange(ix.p_prime), probe_radius, trace=tr)
                if yes:
                    out.append(int(u))
            else:
                out.append(int(u))
    return np.asarray(sorted(out), dtype=np.int64)
