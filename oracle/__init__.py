"""FP64 CPU oracle for RkMIPS and for the steps of SAH.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the
benchmark may import this package; the library under ``paper_2211_12751_gb300`` never
does, and this package never imports it.  The two share no code.

* ``oracle.c`` (compiled here with gcc, -O2 -fopenmp -ffp-contract=off) is the plain
  definition of RkMIPS (Def. 1) written out as a brute-force count in double precision.
* ``oracle.sah`` restates the paper's algorithms step by step in numpy FP64 for small
  inputs: SAT (Eq. 6-8), SRP hashing (Eq. 1, Eq. 9), SA-ALSH indexing and query
  (Alg. 1, Alg. 2), Cone-Tree construction (Alg. 3), the node- and vector-level upper
  bounds (Lemma 2, Lemma 3), SAH indexing (Alg. 4) and the SAH query (Alg. 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (host C, no GPU)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64, I32 = ctypes.c_int64, ctypes.c_int32
            lib.oracle_threads.restype = I32
            lib.oracle_set_threads.argtypes = [I32]
            lib.oracle_scores.argtypes = [P, I64, P, I64, I32, P]
            lib.oracle_query_scores.argtypes = [P, I64, I32, P, I64, P]
            lib.oracle_count_above.argtypes = [P, I64, P, I64, I32, P, P, I64, P]
            lib.oracle_rkmips.argtypes = [P, I64, P, I64, I32, P, I32, P]
            lib.oracle_rkmips.restype = I64
            lib.oracle_tau.argtypes = [P, I64, P, I64, I32, I32, P, I64, P]
            lib.oracle_rkmips_tau.argtypes = [P, I64, I32, P, I32, P, I32, P]
            lib.oracle_rkmips_tau.restype = I64
            lib.oracle_margins.argtypes = [P, I32, P, I32, P, I32, P, I64, P]
            _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(_load().oracle_threads())


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def scores(U, P) -> np.ndarray:
    """All <u,p> in FP64 (m x n); tiny inputs only."""
    U, P = _f32(U), _f32(P)
    out = np.empty((U.shape[0], P.shape[0]), dtype=np.float64)
    _load().oracle_scores(_ptr(U), U.shape[0], _ptr(P), P.shape[0], U.shape[1], _ptr(out))
    return out


def query_scores(U, Q) -> np.ndarray:
    """<u,q> in FP64 for every user and query (m x nq)."""
    U, Q = _f32(U), _f32(np.atleast_2d(Q))
    out = np.empty((U.shape[0], Q.shape[0]), dtype=np.float64)
    _load().oracle_query_scores(_ptr(U), U.shape[0], U.shape[1], _ptr(Q), Q.shape[0], _ptr(out))
    return out


def count_above(U, P, q, users=None) -> np.ndarray:
    """c_u(q) = #{p : <u,p> > <u,q>} for the listed users (default: all)."""
    U, P, q = _f32(U), _f32(P), _f32(q).ravel()
    if users is None:
        cnt, uptr = U.shape[0], None
    else:
        users = np.ascontiguousarray(users, dtype=np.int64)
        cnt, uptr = users.shape[0], _ptr(users)
    out = np.empty(cnt, dtype=np.int64)
    _load().oracle_count_above(_ptr(U), U.shape[0], _ptr(P), P.shape[0], U.shape[1], _ptr(q),
                               uptr, cnt, _ptr(out))
    return out


def rkmips(U, P, q, k) -> np.ndarray:
    """RkMIPS(q, k): ascending int32 user ids (Def. 1, ties kept for q)."""
    U, P, q = _f32(U), _f32(P), _f32(q).ravel()
    out = np.empty(U.shape[0], dtype=np.int32)
    r = _load().oracle_rkmips(_ptr(U), U.shape[0], _ptr(P), P.shape[0], U.shape[1], _ptr(q),
                              int(k), _ptr(out))
    return out[:r].copy()


def tau(U, P, kmax, users=None) -> np.ndarray:
    """tau_u(1..kmax): the j-th largest <u,p> over P (-inf past n); rows follow ``users``."""
    U, P = _f32(U), _f32(P)
    if users is None:
        cnt, uptr = U.shape[0], None
    else:
        users = np.ascontiguousarray(users, dtype=np.int64)
        cnt, uptr = users.shape[0], _ptr(users)
    out = np.empty((cnt, int(kmax)), dtype=np.float64)
    _load().oracle_tau(_ptr(U), U.shape[0], _ptr(P), P.shape[0], U.shape[1], int(kmax), uptr, cnt,
                       _ptr(out))
    return out


def rkmips_tau(U, tau_all, q, k) -> np.ndarray:
    """RkMIPS from cached thresholds (tau over all users, k <= kmax)."""
    U, q = _f32(U), _f32(q).ravel()
    tau_all = np.ascontiguousarray(tau_all, dtype=np.float64)
    kmax = tau_all.shape[1]
    assert 1 <= k <= kmax
    out = np.empty(U.shape[0], dtype=np.int32)
    r = _load().oracle_rkmips_tau(_ptr(U), U.shape[0], U.shape[1], _ptr(tau_all), kmax, _ptr(q),
                                  int(k), _ptr(out))
    return out[:r].copy()


def margins(U, tau_rows, q, k, users) -> np.ndarray:
    """|<u,q> - tau_u(k)| / (||u|| ||q||) for the listed users (tau_rows follow ``users``)."""
    U, q = _f32(U), _f32(q).ravel()
    users = np.ascontiguousarray(users, dtype=np.int64)
    tau_rows = np.ascontiguousarray(tau_rows, dtype=np.float64)
    out = np.empty(users.shape[0], dtype=np.float64)
    _load().oracle_margins(_ptr(U), U.shape[1], _ptr(tau_rows), tau_rows.shape[1], _ptr(q), int(k),
                           _ptr(users), users.shape[0], _ptr(out))
    return out


def rkmips_sampled(U, P, q, k, users) -> np.ndarray:
    """Membership of the listed users only (bool per listed user), by the count rule."""
    return count_above(U, P, q, users) < int(k)


def f1(found, truth) -> float:
    """F1 = 2|A n E| / (|A| + |E|), 1 when both are empty (per query)."""
    a, e = set(np.asarray(found).tolist()), set(np.asarray(truth).tolist())
    if not a and not e:
        return 1.0
    return 2.0 * len(a & e) / (len(a) + len(e))
