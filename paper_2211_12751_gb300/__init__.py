"""Python binding of libsah (SAH RkMIPS on one GB300): argument marshalling only.

Every step of the search runs in the CUDA kernels of ``libsah.so`` behind the C-ABI in
``include/sah.h``; this module converts numpy arrays and torch tensors into pointers,
sizes and streams.  It has no compute path of its own: if the library is not built, or
no GPU is present, calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "sah.h")
LIB_PATH = os.path.join(HERE, "_build", "libsah.so")

SAH_OK, SAH_ERR_ARG, SAH_ERR_OOM, SAH_ERR_CUDA = 0, 1, 2, 3
SAH_ERR_BUFFER_TOO_SMALL, SAH_ERR_DEVICE_TIMEOUT, SAH_ERR_BUSY, SAH_ERR_UNSUPPORTED = 4, 5, 6, 7
EXACT, SAALSH = 0, 1
INJECT_USER_PASS, INJECT_VERIFY = 1, 2
FP32, BF16, FP8 = 0, 1, 2
BLOCK_CONE, BLOCK_NORM = 0, 1   # sah_blocking: Cone-Tree leaves, or Simpfer's norm-sorted blocks
SAT, QNF = 0, 1                 # sah_transform: SA-ALSH's SAT (Eq. 6-7) or H2-ALSH's QNF (Eq. 3-4)

_lib = None


class SahError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libsah status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("k_max", ctypes.c_int32),
        ("leaf_size", ctypes.c_int32),
        ("b", ctypes.c_float),
        ("n_tables", ctypes.c_int32),
        ("code_bits", ctypes.c_int32),
        ("p_prime", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("probe_radius", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("srp", ctypes.c_void_p),
        ("tc_user_pass", ctypes.c_int32),
        ("blocking", ctypes.c_int32),
        ("transform", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "n_items", "n_users", "n_blocks", "n_partitions", "device_bytes", "queries",
        "block_pairs_total", "block_pairs_kept", "users_scored", "users_yes_early",
        "survivors", "fp64_rescored", "results", "users_in_kept_blocks", "items_scanned")] + [
        ("stage_ms", ctypes.c_double * 8), ("stage_launches", ctypes.c_int64 * 8),
        ("build_gemm_ms", ctypes.c_double), ("build_overflow_rows", ctypes.c_int64),
        ("pairs_rescored", ctypes.c_int64), ("tc_scores", ctypes.c_int64), ("block_col_pairs", ctypes.c_int64),
        ("tc_rows", ctypes.c_int64), ("cand_blocks", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name.startswith("stage_") else (float(v) if name.endswith("_ms") else int(v))
        return out


def build(force: bool = False, verbose: bool = False) -> str:
    from .build import build as _build
    return _build(force=force, verbose=verbose)


def declared_functions() -> list:
    """Names of the functions include/sah.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sah_[a-z0-9_]+)\s*\(", text)))


def load(path: Optional[str] = None):
    """Loads libsah.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libsah is not built ({path} missing): call build() first")
    lib = ctypes.CDLL(path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.sah_default_params.argtypes = [ctypes.POINTER(Params)]
    lib.sah_default_params.restype = None
    lib.sah_build_index.argtypes = [P, I64, P, I64, I32, I32, ctypes.POINTER(Params), P, ctypes.POINTER(P)]
    lib.sah_build_index.restype = I32
    lib.sah_rkmips.argtypes = [P, P, I32, I32, P, I64, ctypes.POINTER(I64), P]
    lib.sah_rkmips.restype = I32
    lib.sah_rkmips_batch.argtypes = [P, P, I32, P, P, I32, P, I64, P, P]
    lib.sah_rkmips_batch.restype = I32
    lib.sah_index_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.sah_index_stats.restype = I32
    lib.sah_index_blocks.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I32), P, P, P, P]
    lib.sah_index_blocks.restype = I32
    lib.sah_index_set_timing.argtypes = [P, I32]
    lib.sah_index_set_timing.restype = I32
    lib.sah_index_inject_stall.argtypes = [P, I32]
    lib.sah_index_inject_stall.restype = I32
    lib.sah_index_inject_hash_collision.argtypes = [P, I32]
    lib.sah_index_inject_hash_collision.restype = I32
    lib.sah_rkmips_bruteforce_noalloc.argtypes = [P, I64, P, I64, I32, P, I32, P, I64, P, P]
    lib.sah_rkmips_bruteforce_noalloc.restype = I32
    lib.sah_kmips.argtypes = [P, P, I32, I32, I32, P, P, P]
    lib.sah_kmips.restype = I32
    lib.sah_server_start.argtypes = [P, I32, I32, I32, I64, ctypes.POINTER(P)]
    lib.sah_server_start.restype = I32
    lib.sah_server_submit.argtypes = [P, P, I32, I32, ctypes.POINTER(ctypes.c_uint64)]
    lib.sah_server_submit.restype = I32
    lib.sah_server_poll.argtypes = [P, ctypes.c_uint64, P, I64, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_double)]
    lib.sah_server_poll.restype = I32
    lib.sah_server_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                    ctypes.POINTER(I64)]
    lib.sah_server_info.restype = I32
    lib.sah_server_stop.argtypes = [P]
    lib.sah_server_stop.restype = I32
    lib.sah_selftest_f2d.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    lib.sah_selftest_f2d.restype = I32
    lib.sah_free_index.argtypes = [P]
    lib.sah_free_index.restype = None
    lib.sah_status_string.argtypes = [I32]
    lib.sah_status_string.restype = ctypes.c_char_p
    lib.sah_last_error.argtypes = []
    lib.sah_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != SAH_OK:
        lib = load()
        raise SahError(status, (lib.sah_last_error() or b"").decode() or
                       lib.sah_status_string(status).decode())


def default_params(**kw) -> Params:
    p = Params()
    load().sah_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _host_f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


NOALLOC_MAX_USERS = 1 << 22


def rkmips_bruteforce_noalloc(U, P, q, k: int, out_ids, out_count, m: Optional[int] = None, stream=None):
    """Exact RkMIPS for one query with no allocation anywhere (device tensors in and out):
    U (m x d), P (n x d), q (d) float32; out_ids int32 (capacity = numel); out_count int64
    (one element).  Queued on the stream; read out_count after synchronising.  The tensors
    are only checked here (dtype, layout, device, shapes), never copied or converted: a
    mismatch raises SahError(SAH_ERR_ARG).  ``m`` overrides the user count (at most
    U.shape[0]), e.g. to probe the size limit."""
    import torch

    def bad(msg):
        raise SahError(SAH_ERR_ARG, "rkmips_bruteforce_noalloc: " + msg)

    for name, t, dt in (("U", U, torch.float32), ("P", P, torch.float32), ("q", q, torch.float32),
                        ("out_ids", out_ids, torch.int32), ("out_count", out_count, torch.int64)):
        if not _is_torch(t) or not t.is_cuda:
            bad(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            bad(f"{name} must be {dt}, not {t.dtype}")
        if not t.is_contiguous():
            bad(f"{name} must be contiguous")
    if U.dim() != 2 or P.dim() != 2 or P.shape[1] != U.shape[1]:
        bad("U and P must be 2-D with the same number of columns")
    d = U.shape[1]
    if q.numel() != d:
        bad("q must hold d values")
    if out_count.numel() < 1:
        bad("out_count must hold one value")
    if len({U.device, P.device, q.device, out_ids.device, out_count.device}) != 1:
        bad("all tensors must be on one device")
    lib = load()
    if m is None:
        m = U.shape[0]
    elif m > U.shape[0] and m <= NOALLOC_MAX_USERS:
        bad("m exceeds the rows of U")
    _check(lib.sah_rkmips_bruteforce_noalloc(U.data_ptr(), m, P.data_ptr(), P.shape[0], d,
                                             q.data_ptr(), int(k), out_ids.data_ptr(), out_ids.numel(),
                                             out_count.data_ptr(), _stream_handle(stream)))


def selftest_f2d() -> int:
    """sah_selftest_f2d: the number of float bit patterns whose double widening by the
    library differs from the GPU's own conversion (0 expected)."""
    n = ctypes.c_uint64(0)
    _check(load().sah_selftest_f2d(ctypes.byref(n)))
    return int(n.value)


class Index:
    """A device-resident SAH index (Alg. 4) over users U (m x d) and items P (n x d)."""

    def __init__(self, U, P, params: Optional[Params] = None, stream=None, **kw):
        lib = load()
        srp = kw.pop("srp_matrix", None)
        if params is None:
            params = default_params(**kw)
        self._keep = []
        if srp is not None:
            srp = _host_f32(srp)
            self._keep.append(srp)
            params.srp = srp.ctypes.data
        handle = ctypes.c_void_p()
        if _is_torch(U):
            assert U.is_cuda and P.is_cuda and U.dtype == P.dtype and str(U.dtype) == "torch.float32"
            U, P = U.contiguous(), P.contiguous()
            m, d = U.shape
            n = P.shape[0]
            st = _check(lib.sah_build_index(U.data_ptr(), m, P.data_ptr(), n, d, 1, ctypes.byref(params),
                                            _stream_handle(stream), ctypes.byref(handle)))
        else:
            U, P = _host_f32(U), _host_f32(P)
            m, d = U.shape
            n = P.shape[0]
            _check(lib.sah_build_index(U.ctypes.data, m, P.ctypes.data, n, d, 0, ctypes.byref(params),
                                       _stream_handle(stream), ctypes.byref(handle)))
        self._h = handle
        self.m, self.n, self.d = int(m), int(n), int(d)
        self.params = params

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().sah_free_index(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rkmips(self, q, k: int, mode: int = EXACT, stream=None) -> np.ndarray:
        """Alg. 5 for one query (host q); ascending user ids."""
        lib = load()
        q = _host_f32(q).ravel()
        assert q.shape[0] == self.d
        cap = self.m
        out = np.empty(cap, dtype=np.int32)
        cnt = ctypes.c_int64()
        _check(lib.sah_rkmips(self._h, q.ctypes.data, int(k), int(mode), out.ctypes.data, cap,
                              ctypes.byref(cnt), _stream_handle(stream)))
        return out[:cnt.value].copy()

    def rkmips_batch(self, Q, ks, modes=None, cap: Optional[int] = None, stream=None):
        """Alg. 5 for a batch from host arrays: returns a list of ascending id arrays."""
        lib = load()
        Q = _host_f32(np.atleast_2d(Q))
        nq = Q.shape[0]
        ks = np.ascontiguousarray(np.broadcast_to(np.asarray(ks, dtype=np.int32), (nq,)))
        mptr = None
        if modes is not None:
            modes = np.ascontiguousarray(np.broadcast_to(np.asarray(modes, dtype=np.int32), (nq,)))
            mptr = modes.ctypes.data
        offs = np.zeros(nq + 1, dtype=np.int64)
        cap = cap if cap is not None else self.m * nq
        out = np.empty(max(cap, 1), dtype=np.int32)
        _check(lib.sah_rkmips_batch(self._h, Q.ctypes.data, nq, ks.ctypes.data, mptr, 0, out.ctypes.data, cap,
                                    offs.ctypes.data, _stream_handle(stream)))
        return [out[offs[j]:offs[j + 1]].copy() for j in range(nq)]

    def rkmips_batch_device(self, Q, ks, out_ids, out_offsets, modes=None, stream=None) -> int:
        """Alg. 5 for a batch held in device tensors (Q float32 nq x d, ks int32, out_ids int32,
        out_offsets int64 nq + 1).  Returns the number of ids written."""
        lib = load()
        nq = Q.shape[0]
        mptr = modes.data_ptr() if modes is not None else None
        st = lib.sah_rkmips_batch(self._h, Q.data_ptr(), nq, ks.data_ptr(), mptr, 1, out_ids.data_ptr(),
                                  out_ids.numel(), out_offsets.data_ptr(), _stream_handle(stream))
        _check(st)
        return int(out_offsets[nq].item()) if nq else 0

    def kmips(self, Q, k: int, stream=None):
        """sah_kmips: the k best items of each row of Q found through the SimHash tables
        (host arrays in, host arrays out): (ids nq x k, -1 past the end; FP32 scores)."""
        Q = _host_f32(Q)
        Q = Q.reshape(-1, self.d) if Q.size else np.zeros((0, self.d), np.float32)
        nq = Q.shape[0]
        ids = np.empty((nq, int(k)), np.int32)
        sc = np.empty((nq, int(k)), np.float32)
        _check(load().sah_kmips(self._h, Q.ctypes.data, nq, int(k), 0, ids.ctypes.data, sc.ctypes.data,
                                _stream_handle(stream)))
        return ids, sc

    def kmips_device(self, Q, k: int, out_ids, out_scores=None, stream=None):
        """sah_kmips with device buffers (torch tensors): Q float32 nq x d, out_ids int32
        nq x k, out_scores float32 nq x k or None."""
        nq = Q.shape[0]
        _check(load().sah_kmips(self._h, Q.data_ptr(), nq, int(k), 1, out_ids.data_ptr(),
                                out_scores.data_ptr() if out_scores is not None else None, _stream_handle(stream)))

    def raw_batch(self, Q, nq, ks, modes, on_device, out_ids, cap, offsets, stream=None) -> int:
        """Direct call of sah_rkmips_batch with raw pointers; returns the status."""
        return load().sah_rkmips_batch(self._h, Q, nq, ks, modes, on_device, out_ids, cap, offsets,
                                       _stream_handle(stream))

    def blocks(self):
        """Cone-Tree leaves: (ids in leaf order, leaf starts, cos theta_u, cos omega)."""
        lib = load()
        mnz, nb = ctypes.c_int64(), ctypes.c_int32()
        _check(lib.sah_index_blocks(self._h, ctypes.byref(mnz), ctypes.byref(nb), None, None, None, None))
        ids = np.empty(mnz.value, np.int32)
        starts = np.empty(nb.value + 1, np.int32)
        ct = np.empty(mnz.value, np.float32)
        cw = np.empty(nb.value, np.float32)
        _check(lib.sah_index_blocks(self._h, ctypes.byref(mnz), ctypes.byref(nb), ids.ctypes.data,
                                    starts.ctypes.data, ct.ctypes.data, cw.ctypes.data))
        return ids, starts, ct, cw

    def inject_stall(self, site: int):
        """sah_index_inject_stall: the next query call's MMA thread at `site` (1: user pass,
        2: kMIPS decision) stops after one tile, so the call returns SAH_ERR_DEVICE_TIMEOUT."""
        _check(load().sah_index_inject_stall(self._h, int(site)))

    def inject_hash_collision(self, enable: bool = True):
        """sah_index_inject_hash_collision: the next query call gives every row one hash, so
        the column table is built again comparing whole vectors; the answers do not change."""
        _check(load().sah_index_inject_hash_collision(self._h, 1 if enable else 0))

    def set_timing(self, enable: bool = True):
        _check(load().sah_index_set_timing(self._h, 1 if enable else 0))

    def stats(self) -> dict:
        s = Stats()
        _check(load().sah_index_stats(self._h, ctypes.byref(s)))
        return s.as_dict()


class Server:
    """Continuous-batching server over an Index (see sah_server_* in include/sah.h)."""

    def __init__(self, index: "Index", max_slots: int = 4096, max_batch: int = 512, workers: int = 2,
                 hbm_budget_bytes: int = 0):
        self._lib = load()
        self.index = index
        h = ctypes.c_void_p()
        _check(self._lib.sah_server_start(index._h, max_slots, max_batch, workers, hbm_budget_bytes,
                                          ctypes.byref(h)))
        self._h = h
        self._buf = np.empty(index.m, dtype=np.int32)

    def submit(self, q, k: int, mode: int = EXACT) -> int:
        q = _host_f32(q).ravel()
        t = ctypes.c_uint64()
        _check(self._lib.sah_server_submit(self._h, q.ctypes.data, int(k), int(mode), ctypes.byref(t)))
        return int(t.value)

    def try_submit(self, q, k: int, mode: int = EXACT):
        """Like submit, but returns None instead of raising when every slot is taken."""
        q = _host_f32(q).ravel()
        t = ctypes.c_uint64()
        st = self._lib.sah_server_submit(self._h, q.ctypes.data, int(k), int(mode), ctypes.byref(t))
        if st == SAH_ERR_BUSY:
            return None
        _check(st)
        return int(t.value)

    def poll(self, ticket: int):
        """(ids, latency_s) once finished, None while queued or running."""
        cnt = ctypes.c_int64()
        lat = ctypes.c_double()
        st = self._lib.sah_server_poll(self._h, ticket, self._buf.ctypes.data, self._buf.shape[0],
                                       ctypes.byref(cnt), ctypes.byref(lat))
        if st == SAH_ERR_BUSY:
            return None
        _check(st)
        return self._buf[:cnt.value].copy(), lat.value

    def info(self) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        _check(self._lib.sah_server_info(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("batches", "batched_requests", "max_batch_seen", "split_ticks"), [x.value for x in v]))

    def stop(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.sah_server_stop(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
