"""Seeded synthetic workloads for RkMIPS (items P, users U, queries Q, k values).

This module only draws random numbers and shapes them into the workloads' value
distributions.  It holds none of the method's arithmetic: no inner products, no
thresholds, no bounds, no hashing.  Both the FP64 oracle (``oracle/``) and the CUDA
library read what it returns, which is why it lives in a module of its own.

Recipes (the paper's real datasets are matrix-factorisation embeddings with d = 100,
and its queries are item vectors drawn from P; see the Experiments section, "Setup",
and the appendix "Procedure for Dataset Generation"):

* ``gauss``  - entries i.i.d. N(0,1); each row rescaled to norm exp(N(0, sigma^2)).
* ``mf``     - a shared rank-50 factor matrix W (50 x d, entries N(0,1)/sqrt(50));
               rows are G @ W with G ~ N(0,1)^(rows x 50); rows rescaled to norm
               exp(N(0, sigma^2)); a fraction ``boost_frac`` of the items, chosen
               uniformly, get their norm multiplied by ``boost``.

Draw order inside one workload: W (mf only), then P, then U, then the query indices,
then the k values.  Everything is float32 and C-contiguous.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

__all__ = ["Workload", "make", "CONFIGS", "srp_matrix", "tie_case", "poisson_arrivals"]


@dataclasses.dataclass
class Workload:
    name: str
    P: np.ndarray            # n x d float32, items
    U: np.ndarray            # m x d float32, users
    query_idx: np.ndarray    # nq int64, rows of P used as queries
    ks: np.ndarray           # k values (either one per query, or the set every query runs at)
    every_k: bool            # True: every query is asked at every k in ``ks``
    recipe: dict

    @property
    def Q(self) -> np.ndarray:
        return np.ascontiguousarray(self.P[self.query_idx])

    @property
    def n(self) -> int:
        return self.P.shape[0]

    @property
    def m(self) -> int:
        return self.U.shape[0]

    @property
    def d(self) -> int:
        return self.P.shape[1]

    def requests(self):
        """(query row, k) pairs in the order a batch submits them."""
        Q = self.Q
        if self.every_k:
            qi = np.repeat(np.arange(Q.shape[0]), len(self.ks))
            kk = np.tile(np.asarray(self.ks, dtype=np.int32), Q.shape[0])
        else:
            qi = np.arange(Q.shape[0])
            kk = np.asarray(self.ks, dtype=np.int32)
        return np.ascontiguousarray(Q[qi]), kk.astype(np.int32), qi


def _rescale_rows(X: np.ndarray, target_norm: np.ndarray) -> np.ndarray:
    nrm = np.sqrt(np.einsum("ij,ij->i", X, X, dtype=np.float64))
    nrm[nrm == 0] = 1.0
    return X * (target_norm / nrm)[:, None]


def _gauss_rows(rng, rows, d, sigma):
    X = rng.standard_normal((rows, d))
    return _rescale_rows(X, np.exp(rng.normal(0.0, sigma, rows)))


def _mf_rows(rng, rows, W, sigma, nonneg=False):
    G = rng.standard_normal((rows, W.shape[0]))
    if nonneg:
        G = np.abs(G)
    return _rescale_rows(G @ W, np.exp(rng.normal(0.0, sigma, rows)))


# name -> recipe.  Sizes follow the five benchmark configurations.
CONFIGS = {
    "c1": dict(kind="gauss", n=1000, m=2000, d=16, sigma=0.5, nq=10, ks=[10], every_k=True),
    "c2": dict(kind="mf", n=17770, m=480000, d=50, sigma=0.7, boost_frac=0.05, boost=3.0,
               nq=100, ks=[1, 5, 10, 20, 50], every_k=True),
    "c3": dict(kind="mf", n=100000, m=1000000, d=64, sigma=0.7, boost_frac=0.05, boost=3.0,
               nq=1000, ks=[10, 50], every_k=True),
    "c4": dict(kind="mf", n=100000, m=1000000, d=100, sigma=0.7, boost_frac=0.05, boost=3.0,
               nq=10000, ks="uniform1-50", every_k=False),
    "c5": dict(kind="mf", n=1000000, m=2000000, d=128, sigma=0.7, boost_frac=0.05, boost=3.0,
               nq=5000, ks=[10, 50], every_k=True),
}


def make(name: str = "c1", seed: int = 0, **override) -> Workload:
    """Build a workload from a named recipe; keyword overrides change sizes etc.

    ``make("c2", m=20000)`` keeps the C2 value distribution at a smaller size.
    """
    r = dict(CONFIGS[name])
    r.update(override)
    rng = np.random.default_rng(seed)
    n, m, d = int(r["n"]), int(r["m"]), int(r["d"])
    if r["kind"] == "gauss":
        P = _gauss_rows(rng, n, d, r["sigma"])
        U = _gauss_rows(rng, m, d, r["sigma"])
    elif r["kind"] in ("mf", "nmf"):
        # "nmf": non-negative factors (|N(0,1)| entries), like the NMF embeddings the paper's
        # recommendation datasets are made of; "mf": zero-mean factors
        nonneg = r["kind"] == "nmf"
        rank = int(r.get("rank", 50))
        W = rng.standard_normal((rank, d)) / np.sqrt(rank)
        if nonneg:
            W = np.abs(W)
        P = _mf_rows(rng, n, W, r["sigma"], nonneg)
        nb = int(round(r["boost_frac"] * n))
        if nb:
            boosted = rng.choice(n, size=nb, replace=False)
            P[boosted] *= r["boost"]
        U = _mf_rows(rng, m, W, r["sigma"], nonneg)
    else:
        raise ValueError(r["kind"])
    nq = min(int(r["nq"]), n)
    query_idx = np.sort(rng.choice(n, size=nq, replace=False)).astype(np.int64)
    ks = r["ks"]
    if isinstance(ks, str):
        assert ks == "uniform1-50"
        ks = rng.integers(1, 51, size=nq)
    ks = np.asarray(ks, dtype=np.int32)
    return Workload(name=name, P=np.ascontiguousarray(P, dtype=np.float32),
                    U=np.ascontiguousarray(U, dtype=np.float32), query_idx=query_idx,
                    ks=ks, every_k=bool(r["every_k"]), recipe=dict(r, seed=seed))


def srp_matrix(rows: int, dim: int, seed: int = 12345) -> np.ndarray:
    """Gaussian projection vectors for Sign Random Projection (Eq. 1): rows x dim, N(0,1)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((rows, dim)), dtype=np.float32)


def tie_case(n: int, m: int, d: int, lo: int = -2, hi: int = 2, seed: int = 0):
    """Small integer-valued P, U, q: every score is exact in FP32 and FP64, ties are common."""
    rng = np.random.default_rng(seed)
    P = rng.integers(lo, hi + 1, size=(n, d)).astype(np.float32)
    U = rng.integers(lo, hi + 1, size=(m, d)).astype(np.float32)
    q = rng.integers(lo, hi + 1, size=(d,)).astype(np.float32)
    return P, U, q


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 1) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def random_k(count: int, kmax: int = 50, seed: int = 2, kmin: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(kmin, kmax + 1, size=count).astype(np.int32)


def sample_rows(total: int, count: int, seed: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(total, size=min(count, total), replace=False)).astype(np.int64)


def maybe_subsample(W: Workload, users: Optional[np.ndarray]) -> np.ndarray:
    return W.U if users is None else np.ascontiguousarray(W.U[users])
