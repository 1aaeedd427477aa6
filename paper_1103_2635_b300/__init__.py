"""Python binding of librbc.so: exact nearest-neighbour search with the
Random Ball Cover on one B300 (sm_103a).

Argument marshalling only.  Every step of every search runs in the library's
CUDA kernels; this module passes pointers, sizes and the caller's stream.

Arrays may be torch CUDA tensors (device pointers; the call is stream-ordered
on ``torch.cuda.current_stream()`` unless a stream is given) or numpy arrays
(host pointers; the library copies to and from the device inside the call).

    import paper_1103_2635_b300 as rbc
    ids, dist = rbc.bf_search(Q, X, k=10)                       # BF(Q, X)
    index = rbc.rbc_build(X, n_r=1024, storage=rbc.BF16)        # R, lists, radii
    ids, dist = rbc.rbc_search(index, Q, k=10)                  # exact search

The library must have been built (``python -m paper_1103_2635_b300.build_lib``
or ``__graft_entry__.build()``); importing without it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "L2", "L1", "EXACT", "ONESHOT", "F32", "BF16", "F16", "FP8E4M3", "PLAN_WINDOW", "PLAN_TILE_UNION",
    "PLAN_WINDOW_OFFSET",
    "RbcError", "bf_search", "bf_search_noalloc", "rbc_build", "rbc_search", "rbc_sample_reps",
    "RbcIndex", "last_stats", "set_timing", "trim_workspace", "library_path", "load",
    "search_workspace", "plan_batch", "Server", "Group",
]

L2, L1 = 0, 1
EXACT, ONESHOT = 0, 1
F32, BF16, F16, FP8E4M3 = 0, 1, 2, 3
PLAN_WINDOW, PLAN_TILE_UNION, PLAN_WINDOW_OFFSET = 0, 1, 2
_STATUS = {0: "ok", -1: "invalid argument", -2: "out of device memory", -3: "CUDA error",
           -4: "device wait timed out", -5: "unsupported"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "librbc.so")
_lib = None


class RbcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("mode", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("rerank_c", ctypes.c_int32), ("plan", ctypes.c_int32),
                ("rep_ids", ctypes.c_void_p)]


class _Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("n_r", ctypes.c_int32),
                ("s", ctypes.c_int32), ("metric", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("list_entries", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("device", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "queries", "kept_reps", "tile_points", "stage2_items", "uncertified", "fp64_ties",
        "boundary_ties", "pairs", "kernel_launches")] + [
        (name, ctypes.c_double) for name in ("stage1_ms", "stage2_ms", "select_ms", "fallback_ms")] + [
        ("candidates", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64)]


class _GroupedStats(ctypes.Structure):
    _fields_ = [("indexes", ctypes.c_int64), ("rows", ctypes.c_int64),
                ("representatives", ctypes.c_int64), ("dim", ctypes.c_int32),
                ("work_item_points", ctypes.c_int32), ("queries", ctypes.c_int64),
                ("tiles", ctypes.c_int64), ("work_items", ctypes.c_int64),
                ("uncertified", ctypes.c_int64), ("fp64_ties", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64), ("device_errors", ctypes.c_uint32)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("k_max", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("hbm_budget", ctypes.c_int64)]


class _RequestInfo(ctypes.Structure):
    _fields_ = [("t_submit_ns", ctypes.c_int64), ("t_start_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64), ("batch", ctypes.c_int64),
                ("batch_queries", ctypes.c_int64), ("batch_requests", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class _ServingStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in ("requests", "queries", "batches")] + [
        (name, ctypes.c_double) for name in (
            "p50_ms", "p99_ms", "mean_ms", "max_ms", "queue_p50_ms", "queue_p99_ms", "wall_s",
            "queries_per_s", "mean_batch_queries")] + [
        ("peak_reserved_bytes", ctypes.c_int64), ("hbm_budget", ctypes.c_int64),
        ("max_in_flight", ctypes.c_int32), ("workers", ctypes.c_int32)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load librbc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(
            f"{_LIB_PATH} is missing: build it with `python -m paper_1103_2635_b300.build_lib`"
        )
    lib = ctypes.CDLL(_LIB_PATH)
    P, I64, I32, U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    lib.rbc_sample_reps.argtypes = [I64, I32, U64, P]
    lib.bf_search.argtypes = [P, I64, P, I64, I32, I32, I32, I32, P, P, P]
    lib.bf_search_noalloc.argtypes = [P, I64, P, I64, I32, I32, I32, P, P, P]
    lib.rbc_build.argtypes = [P, I64, I32, I32, I32, I32, ctypes.POINTER(_Opts), P,
                              ctypes.POINTER(ctypes.c_void_p)]
    lib.rbc_search.argtypes = [P, P, I64, I32, P, P, P]
    lib.rbc_search_check.argtypes = [P, P]
    lib.rbc_index_info.argtypes = [P, ctypes.POINTER(_Desc)]
    lib.rbc_index_export.argtypes = [P, P, P, P, P]
    lib.rbc_last_stats.argtypes = [ctypes.POINTER(_Stats)]
    lib.rbc_set_timing.argtypes = [ctypes.c_int]
    lib.rbc_set_timing.restype = ctypes.c_int
    lib.rbc_free.argtypes = [P]
    lib.rbc_free.restype = None
    lib.rbc_trim_workspace.argtypes = []
    lib.rbc_last_error.restype = ctypes.c_char_p
    lib.rbc_default_opts.argtypes = [ctypes.POINTER(_Opts)]
    lib.rbc_default_opts.restype = None
    lib.rbc_search_workspace.argtypes = [P, I64, I32, ctypes.POINTER(I64)]
    lib.rbc_plan_batch.argtypes = [P, P, I32, I64, I64, I64, I64, I64]
    lib.rbc_server_create.argtypes = [P, ctypes.POINTER(_ServerOpts), ctypes.POINTER(ctypes.c_void_p)]
    lib.rbc_server_submit.argtypes = [P, P, I64, I32, P, P, ctypes.POINTER(U64)]
    lib.rbc_server_wait.argtypes = [P, U64, I64, ctypes.POINTER(_RequestInfo)]
    lib.rbc_server_stats.argtypes = [P, I32, ctypes.POINTER(_ServingStats)]
    lib.rbc_server_destroy.argtypes = [P]
    lib.rbc_server_destroy.restype = None
    lib.rbc_group_create.argtypes = [P, I32, P, ctypes.POINTER(ctypes.c_void_p)]
    lib.rbc_group_search.argtypes = [P, P, P, I32, P, P, P]
    lib.rbc_group_search_split.argtypes = [P, P, P, I32, P, P, P]
    lib.rbc_group_tune.argtypes = [P, P, P, I32, P, ctypes.POINTER(I32)]
    lib.rbc_group_stats.argtypes = [P, ctypes.POINTER(_GroupedStats)]
    lib.rbc_group_free.argtypes = [P]
    lib.rbc_group_free.restype = None
    for f in ("rbc_sample_reps", "bf_search", "bf_search_noalloc", "rbc_build", "rbc_search", "rbc_search_check", "rbc_index_info",
              "rbc_index_export", "rbc_last_stats", "rbc_search_workspace", "rbc_plan_batch",
              "rbc_server_create", "rbc_server_submit", "rbc_server_wait", "rbc_server_stats",
              "rbc_group_create", "rbc_group_search", "rbc_group_search_split", "rbc_group_tune",
              "rbc_group_stats"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise RbcError(rc, load().rbc_last_error().decode())


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _arg(a, dtype):
    """(pointer, keepalive, is_device) for a torch tensor or a numpy-compatible array."""
    if _is_torch(a):
        import torch

        want = {np.float32: torch.float32, np.int64: torch.int64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return a.data_ptr(), a, a.is_cuda
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr, False


def _stream_of(stream, device_side: bool):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    if device_side:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return 0


def _check_out(a, dtype, m: int, k: int):
    """Pointer of a caller's [m, k] output, written in place (no copy)."""
    if tuple(a.shape) != (m, k):
        raise ValueError(f"expected an [{m}, {k}] output, got shape {tuple(a.shape)}")
    p, kept, dev = _arg(a, dtype)
    if kept is not a:
        raise TypeError(f"outputs must be contiguous {np.dtype(dtype).name} arrays")
    return p, dev


def _outputs(m: int, k: int, like_device, out_ids, out_dist):
    if out_ids is None:
        if like_device is not None:
            import torch

            out_ids = torch.empty((m, k), dtype=torch.int64, device=like_device)
            out_dist = torch.empty((m, k), dtype=torch.float32, device=like_device)
        else:
            out_ids = np.empty((m, k), dtype=np.int64)
            out_dist = np.empty((m, k), dtype=np.float32)
    return out_ids, out_dist


def rbc_sample_reps(n: int, n_r: int, seed: int = 0) -> np.ndarray:
    """The library's representative set: n_r distinct ids of [0, n), ascending."""
    out = np.empty(n_r, dtype=np.int64)
    _check(load().rbc_sample_reps(n, n_r, seed, out.ctypes.data))
    return out


def bf_search(Q, X, k: int, metric: int = L2, storage: int = F32, out_ids=None, out_dist=None,
              stream=None):
    """BF(Q, X): ids [m, k] int64 and rho [m, k] float32, sorted by (rho, id)."""
    qp, qk, qdev = _arg(Q, np.float32)
    xp, xk, xdev = _arg(X, np.float32)
    m, d = qk.shape
    n = xk.shape[0]
    if xk.shape[1] != d:
        raise ValueError("Q and X differ in dimension")
    out_ids, out_dist = _outputs(m, k, qk.device if qdev else None, out_ids, out_dist)
    ip, _, idev = _arg(out_ids, np.int64)
    dp, _, ddev = _arg(out_dist, np.float32)
    st = _stream_of(stream, qdev or xdev or idev)
    _check(load().bf_search(qp, m, xp, n, d, k, metric, storage, ip, dp, st))
    return out_ids, out_dist


def bf_search_noalloc(Q, X, k: int, metric: int = L2, out_ids=None, out_dist=None, stream=None):
    """BF(Q, X) in FP32 without any device allocation (library-owned static
    scratch; device tensors only; calls must not overlap on the GPU)."""
    qp, qk, qdev = _arg(Q, np.float32)
    xp, xk, _ = _arg(X, np.float32)
    m, d = qk.shape
    out_ids, out_dist = _outputs(m, k, qk.device if qdev else None, out_ids, out_dist)
    ip, _, _ = _arg(out_ids, np.int64)
    dp, _, _ = _arg(out_dist, np.float32)
    st = _stream_of(stream, qdev)
    _check(load().bf_search_noalloc(qp, m, xp, xk.shape[0], d, k, metric, ip, dp, st))
    return out_ids, out_dist


class RbcIndex:
    """A built Random Ball Cover (library-owned device memory)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        d = _Desc()
        _check(load().rbc_index_info(self._h, ctypes.byref(d)))
        return {f: getattr(d, f) for f, _ in _Desc._fields_}

    def export(self) -> dict:
        """reps, list offsets, list members (ids), radii -- host numpy arrays."""
        inf = self.info()
        reps = np.empty(inf["n_r"], np.int64)
        off = np.empty(inf["n_r"] + 1, np.int64)
        mem = np.empty(inf["list_entries"], np.int64)
        psi = np.empty(inf["n_r"], np.float32)
        _check(load().rbc_index_export(self._h, reps.ctypes.data, off.ctypes.data, mem.ctypes.data,
                                       psi.ctypes.data))
        return {"reps": reps, "offsets": off, "members": mem, "psi": psi}

    def search(self, Q, k: int, out_ids=None, out_dist=None, stream=None):
        return rbc_search(self, Q, k, out_ids=out_ids, out_dist=out_dist, stream=stream)

    def close(self):
        if self._h is not None and self._h.value:
            load().rbc_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rbc_build(X, n_r: int, metric: int = L2, seed: int = 0, mode: int = EXACT,
              storage: int = F32, s: int = 0, rerank_c: int = 0, rep_ids=None,
              plan: int = PLAN_WINDOW, stream=None) -> RbcIndex:
    """Build the Random Ball Cover of X (Sections 4-5 of the paper).  ``plan``
    picks the exact search's stage two for bf16 / fp16 storage."""
    xp, xk, xdev = _arg(X, np.float32)
    n, d = xk.shape
    opts = _Opts()
    load().rbc_default_opts(ctypes.byref(opts))
    opts.seed, opts.mode, opts.storage, opts.rerank_c = seed, mode, storage, rerank_c
    opts.plan = plan
    keep = None
    if rep_ids is not None:
        keep = np.ascontiguousarray(rep_ids, dtype=np.int64)
        opts.rep_ids = keep.ctypes.data
    h = ctypes.c_void_p()
    st = _stream_of(stream, xdev)
    _check(load().rbc_build(xp, n, d, n_r, s, metric, ctypes.byref(opts), st, ctypes.byref(h)))
    return RbcIndex(h.value)


def rbc_search(index: RbcIndex, Q, k: int, out_ids=None, out_dist=None, stream=None):
    """k-NN of every query with the index: ids [m, k], rho [m, k].  Exact
    mode returns the exact k nearest neighbours (Section 5.2); one-shot mode
    the k nearest within the list of the query's nearest representative
    (Section 5.1)."""
    qp, qk, qdev = _arg(Q, np.float32)
    m = qk.shape[0]
    out_ids, out_dist = _outputs(m, k, qk.device if qdev else None, out_ids, out_dist)
    ip, _, idev = _arg(out_ids, np.int64)
    dp, _, _ = _arg(out_dist, np.float32)
    st = _stream_of(stream, qdev or idev)
    _check(load().rbc_search(index.handle, qp, m, k, ip, dp, st))
    return out_ids, out_dist


def search_check(index: RbcIndex, stream=None) -> None:
    """Wait for the stream, then raise if a search recorded under stream
    capture (a CUDA graph) left device error flags in the index."""
    _check(load().rbc_search_check(index.handle, _stream_of(stream, True)))


def trim_workspace() -> None:
    """Release the search workspace cached for the current device."""
    _check(load().rbc_trim_workspace())


def set_timing(on: bool) -> bool:
    """Per-phase device timing of later searches on this thread (see last_stats)."""
    return bool(load().rbc_set_timing(1 if on else 0))


def last_stats() -> dict:
    """Counters of this thread's last search call (waits for its stream)."""
    s = _Stats()
    _check(load().rbc_last_stats(ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in _Stats._fields_}


def search_workspace(index: RbcIndex, m: int, k: int) -> int:
    """Upper bound of the device workspace bytes one rbc_search of m queries holds."""
    b = ctypes.c_int64(0)
    _check(load().rbc_search_workspace(index.handle, m, k, ctypes.byref(b)))
    return b.value


def plan_batch(m, k, max_batch: int, mem_left: int, fixed_bytes: int = 0,
               bytes_per_query: int = 0, bytes_per_query_k: int = 0) -> int:
    """The serving engine's admission rule (host only): how many of the queued
    requests (sizes m, neighbour counts k, arrival order) one batch takes."""
    ma = np.ascontiguousarray(m, dtype=np.int64)
    ka = np.ascontiguousarray(k, dtype=np.int32)
    rc = load().rbc_plan_batch(ma.ctypes.data, ka.ctypes.data, len(ma), max_batch, mem_left,
                               fixed_bytes, bytes_per_query, bytes_per_query_k)
    if rc < 0:
        _check(rc)
    return rc


class Server:
    """Continuous-batching request loop over a resident index (rbc_server_*).

    ``submit`` queues a request and returns a ticket at once; the library's
    worker threads merge waiting requests into batches admitted by an HBM
    budget and run them concurrently on their own CUDA streams.  Inputs and
    outputs of a request must stay alive until ``wait`` returns for it; the
    object keeps references to them until then.
    """

    def __init__(self, index: RbcIndex, workers: int = 2, max_batch: int = 16384,
                 k_max: int = 10, hbm_budget: int = 0):
        o = _ServerOpts(workers, max_batch, k_max, 0, hbm_budget)
        h = ctypes.c_void_p()
        _check(load().rbc_server_create(index.handle, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._index = index  # the index must outlive the server
        self._keep = {}
        self.d = index.info()["d"]

    def submit(self, Q, k: int, out_ids=None, out_dist=None) -> int:
        """Queue the queries Q [m, d]; results go to out_ids / out_dist [m, k]
        (allocated as host arrays when omitted).  Returns the ticket."""
        qp, qk, _ = _arg(Q, np.float32)
        m = qk.shape[0] if qk.ndim == 2 else 0
        out_ids, out_dist = _outputs(m, k, None, out_ids, out_dist)
        ip, ik, _ = _arg(out_ids, np.int64)
        dp, dk, _ = _arg(out_dist, np.float32)
        t = ctypes.c_uint64(0)
        _check(load().rbc_server_submit(self._h, qp, m, k, ip, dp, ctypes.byref(t)))
        self._keep[t.value] = (qk, ik, dk)
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1):
        """(out_ids, out_dist, info) of a finished request; raises RbcError on
        its error or when it is still running after timeout_us."""
        info = _RequestInfo()
        rc = load().rbc_server_wait(self._h, ticket, timeout_us, ctypes.byref(info))
        if rc == -4 and timeout_us >= 0:
            _check(rc)
        _, ik, dk = self._keep.pop(ticket, (None, None, None))
        _check(rc)
        return ik, dk, {f: getattr(info, f) for f, _ in _RequestInfo._fields_}

    def stats(self, reset: bool = False) -> dict:
        st = _ServingStats()
        _check(load().rbc_server_stats(self._h, int(reset), ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in _ServingStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().rbc_server_destroy(self._h)
        self._h = None
        self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Many exact indexes searched together (rbc_group_*): one resident
    concatenated layout, one persistent tensor-core launch for the stage two
    of every index, each batch shape captured once as a CUDA graph."""

    def __init__(self, indexes, stream=None):
        arr = (ctypes.c_void_p * len(indexes))(*[ix.handle.value for ix in indexes])
        h = ctypes.c_void_p()
        _check(load().rbc_group_create(arr, len(indexes), _stream_of(stream, True), ctypes.byref(h)))
        self._h = h
        self.dims = [ix.info()["d"] for ix in indexes]

    def _pack(self, Qs):
        if len(Qs) != len(self.dims):
            raise ValueError("one query array per index")
        m = np.array([q.shape[0] for q in Qs], dtype=np.int64)
        if all(_is_torch(q) and q.is_cuda for q in Qs):
            import torch

            flat = torch.cat([q.reshape(-1) for q in Qs]).contiguous()
            dev = flat.device
        else:
            flat = np.ascontiguousarray(np.concatenate([np.asarray(q, np.float32).reshape(-1) for q in Qs]))
            dev = None
        return flat, m, dev

    def search(self, Qs, k: int, out_ids=None, out_dist=None, stream=None):
        """Qs: one [m_i, d_i] float32 array per index (all CUDA tensors, or
        host arrays).  Returns ([m_i, k] ids, [m_i, k] rho) per index: views
        of one [sum m_i, k] pair, out_ids / out_dist when given (int64 and
        float32, host or device, e.g. pinned host tensors).  Host arrays are
        passed one pointer per index (rbc_group_search_split), so they are
        copied to the device as they are, with no packing here."""
        if len(Qs) != len(self.dims):
            raise ValueError("one query array per index")
        if (out_ids is None) != (out_dist is None):
            raise ValueError("give both out_ids and out_dist, or neither")
        if all(_is_torch(q) and q.is_cuda for q in Qs):
            flat, m, dev = self._pack(Qs)
            M = int(m.sum())
            ids, dist = _outputs(M, k, dev, out_ids, out_dist)
            ip, _ = _check_out(ids, np.int64, M, k)
            dp, _ = _check_out(dist, np.float32, M, k)
            _check(load().rbc_group_search(self._h, flat.data_ptr(), m.ctypes.data, k, ip, dp,
                                           _stream_of(stream, True)))
        else:
            keep = [_arg(q, np.float32) for q in Qs]
            if any(dev for _, _, dev in keep):
                raise TypeError("queries must be all CUDA tensors or all host arrays")
            for (_, kq, _), d in zip(keep, self.dims):
                if len(kq.shape) != 2 or kq.shape[1] != d:
                    raise ValueError(f"expected [m, {d}] queries, got shape {tuple(kq.shape)}")
            m = np.array([kq.shape[0] for _, kq, _ in keep], dtype=np.int64)
            ptrs = (ctypes.c_void_p * len(keep))(*[p for p, _, _ in keep])
            M = int(m.sum())
            ids, dist = _outputs(M, k, None, out_ids, out_dist)
            ip, idev = _check_out(ids, np.int64, M, k)
            dp, _ = _check_out(dist, np.float32, M, k)
            _check(load().rbc_group_search_split(self._h, ptrs, m.ctypes.data, k, ip, dp,
                                                 _stream_of(stream, idev)))
        cut = np.concatenate([[0], np.cumsum(m)])
        return ([ids[cut[i]:cut[i + 1]] for i in range(len(m))],
                [dist[cut[i]:cut[i + 1]] for i in range(len(m))])

    def tune(self, Qs, k: int, stream=None) -> int:
        """Autotune the stage-two work-item size on this batch; returns it."""
        flat, m, dev = self._pack(Qs)
        fp = flat.data_ptr() if dev is not None else flat.ctypes.data
        w = ctypes.c_int32(0)
        _check(load().rbc_group_tune(self._h, fp, m.ctypes.data, k, _stream_of(stream, dev is not None),
                                     ctypes.byref(w)))
        return w.value

    def stats(self) -> dict:
        st = _GroupedStats()
        _check(load().rbc_group_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in _GroupedStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().rbc_group_free(self._h)
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
