"""Thin ctypes binding of the C ABI in ``include/fec.h`` (``libfec.so``).

Argument marshalling only: every step of the clustering runs in the CUDA
library.  There is no CPU fallback; if the library is missing this module
raises on first use.  Functions keep the C names (``fec_create``,
``fec_cluster``, ``fec_cluster_batch``, ``fec_serve_submit``,
``fec_serve_poll``, ``fec_serve_poll_timed``, ``fec_serve_submit_deadline``,
``fec_serve_get_stats``, ``fec_get_stats``, ``fec_workspace_bytes``,
``fec_set_iteration_caps``, ``fec_status_string``, ``fec_destroy``) and take raw pointers like the C ABI;
``Context`` adds array conveniences on top (numpy arrays = host memory,
torch CUDA tensors = device memory).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

INT64_MAX = (1 << 63) - 1
FEC_MAX_POINTS = 1 << 30

STATUS = {0: "FEC_OK", 1: "FEC_ERR_INVALID_ARG", 2: "FEC_ERR_NONFINITE", 3: "FEC_ERR_OUT_OF_RANGE",
          4: "FEC_ERR_OOM", 5: "FEC_ERR_CUDA", 6: "FEC_ERR_NOT_CONVERGED", 7: "FEC_ERR_NOT_READY",
          8: "FEC_ERR_BUSY", 9: "FEC_ERR_TIMEOUT", 10: "FEC_ERR_INTERNAL"}
FEC_OK, FEC_ERR_NOT_READY, FEC_ERR_TIMEOUT = 0, 7, 9

# Every function the header declares (checked by the CPU tests against include/fec.h).
EXPORTS = ("fec_create", "fec_destroy", "fec_cluster", "fec_cluster_batch", "fec_serve_submit",
           "fec_serve_poll", "fec_serve_poll_timed", "fec_get_stats", "fec_workspace_bytes", "fec_status_string",
           "fec_trace_enable", "fec_trace_read", "fec_cluster_noalloc", "fec_set_iteration_caps",
           "fec_serve_submit_deadline", "fec_serve_get_stats")
FEC_NOALLOC_MAX_POINTS = 32768
FEC_DEFAULT_WAIT_CAP = 1 << 22
FEC_DEFAULT_UNION_CAP = 1 << 20


class FecError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = int(code)
        self.name = STATUS.get(self.code, f"FEC_ERR_UNKNOWN({code})")
        super().__init__(f"{where}: {self.name}" if where else self.name)


class fec_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t),
                ("cuda_stream", ctypes.c_void_p), ("autotune_cache", ctypes.c_char_p)]


class fec_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("cells", ctypes.c_int64), ("subcells", ctypes.c_int64),
                ("num_clusters", ctypes.c_int64), ("key_bits", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("R", ctypes.c_int32), ("h", ctypes.c_int32),
                ("T2", ctypes.c_int64), ("pair_checks", ctypes.c_int64),
                ("pair_box_joins", ctypes.c_int64), ("pair_point_tests", ctypes.c_int64),
                ("pair_same_root", ctypes.c_int64), ("point_evals", ctypes.c_int64),
                ("pairs_queued", ctypes.c_int64), ("boundary_edges", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fec_serve_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "submitted", "completed", "rejected", "expired", "queued", "queue_max", "queue_wait_ns_sum",
        "queue_wait_ns_max", "run_ns_sum", "run_ns_max", "arena_bytes")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fec_trace_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_lib = None


def debug_library() -> bool:
    """True when the environment selects the bounds-checked debug build
    (FEC_LIBRARY=debug; for debugging and its own tests only)."""
    return os.environ.get("FEC_LIBRARY", "") == "debug"


def library_path() -> str:
    return _build.LIB_DEBUG if debug_library() else _build.LIB


def load(build_if_missing: bool = False):
    """Load libfec.so, or libfec_debug.so when FEC_LIBRARY=debug (optionally
    building it first).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        _build.build(debug=debug_library())
    lib = ctypes.CDLL(path)
    vp, i64, i32p, f32p = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p
    lib.fec_create.argtypes = [ctypes.POINTER(fec_options), ctypes.POINTER(vp)]
    lib.fec_create.restype = ctypes.c_int
    lib.fec_destroy.argtypes = [vp]
    lib.fec_destroy.restype = None
    lib.fec_cluster.argtypes = [vp, f32p, i64, ctypes.c_float, i64, i64, vp, i32p]
    lib.fec_cluster.restype = ctypes.c_int
    lib.fec_cluster_batch.argtypes = [vp, f32p, vp, ctypes.c_int32, vp, vp, vp, vp, vp]
    lib.fec_cluster_batch.restype = ctypes.c_int
    lib.fec_serve_submit.argtypes = [vp, f32p, i64, ctypes.c_float, i64, i64, vp,
                                     ctypes.POINTER(ctypes.c_uint64)]
    lib.fec_serve_submit.restype = ctypes.c_int
    lib.fec_serve_submit_deadline.argtypes = [vp, f32p, i64, ctypes.c_float, i64, i64, vp, i64,
                                              ctypes.POINTER(ctypes.c_uint64)]
    lib.fec_serve_submit_deadline.restype = ctypes.c_int
    lib.fec_serve_get_stats.argtypes = [vp, ctypes.POINTER(fec_serve_stats)]
    lib.fec_serve_get_stats.restype = ctypes.c_int
    lib.fec_serve_poll.argtypes = [vp, ctypes.c_uint64, i32p, ctypes.c_int]
    lib.fec_serve_poll.restype = ctypes.c_int
    lib.fec_serve_poll_timed.argtypes = [vp, ctypes.c_uint64, i32p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int64)]
    lib.fec_serve_poll_timed.restype = ctypes.c_int
    lib.fec_get_stats.argtypes = [vp, ctypes.POINTER(fec_stats)]
    lib.fec_get_stats.restype = ctypes.c_int
    lib.fec_workspace_bytes.argtypes = [i64, ctypes.c_float]
    lib.fec_workspace_bytes.restype = i64
    lib.fec_trace_enable.argtypes = [vp, ctypes.c_int]
    lib.fec_trace_enable.restype = ctypes.c_int
    lib.fec_trace_read.argtypes = [vp, ctypes.POINTER(fec_trace_entry), ctypes.c_int]
    lib.fec_trace_read.restype = ctypes.c_int
    lib.fec_cluster_noalloc.argtypes = [f32p, i64, ctypes.c_float, i64, i64, vp, i32p, vp]
    lib.fec_cluster_noalloc.restype = ctypes.c_int
    lib.fec_set_iteration_caps.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32]
    lib.fec_set_iteration_caps.restype = ctypes.c_int
    lib.fec_status_string.argtypes = [ctypes.c_int]
    lib.fec_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


# --------------------------------------------------------------------------
# C-named functions (raw pointers, status codes returned as ints)
# --------------------------------------------------------------------------

def fec_create(device: int = 0, mem_budget_bytes: int = 0, cuda_stream: int = 0,
               autotune_cache: str | None = None) -> int:
    lib = load()
    opt = fec_options(device, mem_budget_bytes, cuda_stream or None,
                      autotune_cache.encode() if autotune_cache else None)
    h = ctypes.c_void_p()
    st = lib.fec_create(ctypes.byref(opt), ctypes.byref(h))
    if st != FEC_OK:
        raise FecError(st, "fec_create")
    return h.value


def fec_destroy(ctx: int) -> None:
    load().fec_destroy(ctx)


def fec_cluster(ctx, xyz_ptr, n, d, min_size, max_size, labels_ptr) -> tuple[int, int]:
    """Returns (status, num_clusters)."""
    k = ctypes.c_int32(-1)
    st = load().fec_cluster(ctx, xyz_ptr, int(n), float(d), int(min_size), int(max_size),
                            labels_ptr, ctypes.byref(k))
    return st, k.value


def fec_cluster_noalloc(xyz_ptr, n, d, min_size, max_size, labels_ptr, cuda_stream=0):
    """Returns (status, num_clusters); no context, no allocation."""
    k = ctypes.c_int32(-1)
    st = load().fec_cluster_noalloc(xyz_ptr, int(n), float(d), int(min_size), int(max_size),
                                    labels_ptr, ctypes.byref(k), cuda_stream or None)
    return st, k.value


def fec_cluster_batch(ctx, xyz_ptr, offsets_ptr, nb, d_ptr, min_ptr, max_ptr, labels_ptr,
                      num_clusters_ptr) -> int:
    return load().fec_cluster_batch(ctx, xyz_ptr, offsets_ptr, int(nb), d_ptr, min_ptr, max_ptr,
                                    labels_ptr, num_clusters_ptr)


def fec_serve_submit(ctx, xyz_ptr, n, d, min_size, max_size, labels_ptr) -> tuple[int, int]:
    t = ctypes.c_uint64(0)
    st = load().fec_serve_submit(ctx, xyz_ptr, int(n), float(d), int(min_size), int(max_size),
                                 labels_ptr, ctypes.byref(t))
    return st, t.value


def fec_serve_submit_deadline(ctx, xyz_ptr, n, d, min_size, max_size, labels_ptr,
                              deadline_us) -> tuple[int, int]:
    t = ctypes.c_uint64(0)
    st = load().fec_serve_submit_deadline(ctx, xyz_ptr, int(n), float(d), int(min_size),
                                          int(max_size), labels_ptr, int(deadline_us),
                                          ctypes.byref(t))
    return st, t.value


def fec_serve_get_stats(ctx) -> dict:
    s = fec_serve_stats()
    st = load().fec_serve_get_stats(ctx, ctypes.byref(s))
    if st != FEC_OK:
        raise FecError(st, "fec_serve_get_stats")
    return s.as_dict()


def fec_serve_poll(ctx, ticket, timeout_ms=-1) -> tuple[int, int]:
    k = ctypes.c_int32(-1)
    st = load().fec_serve_poll(ctx, int(ticket), ctypes.byref(k), int(timeout_ms))
    return st, k.value


def fec_serve_poll_timed(ctx, ticket, timeout_ms=-1) -> tuple[int, int, int]:
    """(status, k, done_ns): done_ns is the CLOCK_MONOTONIC completion time."""
    k = ctypes.c_int32(-1)
    t = ctypes.c_int64(0)
    st = load().fec_serve_poll_timed(ctx, int(ticket), ctypes.byref(k), int(timeout_ms),
                                     ctypes.byref(t))
    return st, k.value, t.value


def fec_get_stats(ctx) -> dict:
    s = fec_stats()
    st = load().fec_get_stats(ctx, ctypes.byref(s))
    if st != FEC_OK:
        raise FecError(st, "fec_get_stats")
    return s.as_dict()


def fec_trace_enable(ctx, enable: bool = True) -> int:
    return load().fec_trace_enable(ctx, 1 if enable else 0)


def fec_trace_read(ctx) -> list:
    """[{name, launches, total_ms}] accumulated since tracing was enabled."""
    lib = load()
    n = lib.fec_trace_read(ctx, None, 0)
    if n <= 0:
        return []
    buf = (fec_trace_entry * n)()
    n = lib.fec_trace_read(ctx, buf, n)
    return [{"name": e.name.decode(), "launches": int(e.launches), "total_ms": float(e.total_ms)}
            for e in buf[:n]]


def fec_set_iteration_caps(ctx, wait_cap: int, union_cap: int) -> int:
    return load().fec_set_iteration_caps(ctx, int(wait_cap), int(union_cap))


def fec_workspace_bytes(n: int, d: float) -> int:
    return int(load().fec_workspace_bytes(int(n), float(d)))


def fec_status_string(status: int) -> str:
    return load().fec_status_string(int(status)).decode()


# --------------------------------------------------------------------------
# Array conveniences
# --------------------------------------------------------------------------

def _ptr(a):
    """Data pointer of a numpy array (host) or a torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_torch(a):
    return type(a).__module__.startswith("torch")


class Context:
    """Owns one fec_ctx.  ``cluster`` accepts numpy (host) or torch arrays."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, cuda_stream: int = 0,
                 autotune_cache: str | None = None):
        self.handle = fec_create(device, mem_budget_bytes, cuda_stream, autotune_cache)

    def close(self):
        if getattr(self, "handle", None):
            fec_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def cluster(self, xyz, d, min_size=1, max_size=INT64_MAX, labels=None):
        """Labels (same kind of array as ``labels``, default: numpy for numpy
        input, a torch tensor on xyz's device for torch input) and k."""
        if _is_torch(xyz):
            import torch
            assert xyz.dtype == torch.float32 and xyz.is_contiguous()
            n = xyz.numel() // 3
            if labels is None:
                labels = torch.empty(n, dtype=torch.int32, device=xyz.device)
        else:
            xyz = np.ascontiguousarray(xyz, dtype=np.float32)
            n = xyz.size // 3
            if labels is None:
                labels = np.empty(n, dtype=np.int32)
        st, k = fec_cluster(self.handle, _ptr(xyz), n, d, min_size, max_size, _ptr(labels))
        if st != FEC_OK:
            raise FecError(st, "fec_cluster")
        return labels, k

    def cluster_batch(self, xyz, offsets, d, min_size, max_size, labels=None):
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        nb = offsets.size - 1
        dd = np.ascontiguousarray(d, dtype=np.float32)
        mn = np.ascontiguousarray(min_size, dtype=np.int64)
        mx = np.ascontiguousarray(max_size, dtype=np.int64)
        ks = np.zeros(max(nb, 1), dtype=np.int32)
        if labels is None:
            if _is_torch(xyz):
                import torch
                labels = torch.empty(int(offsets[-1]), dtype=torch.int32, device=xyz.device)
            else:
                labels = np.empty(int(offsets[-1]), dtype=np.int32)
        if not _is_torch(xyz):
            xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        st = fec_cluster_batch(self.handle, _ptr(xyz), offsets.ctypes.data, nb, dd.ctypes.data,
                               mn.ctypes.data, mx.ctypes.data, _ptr(labels), ks.ctypes.data)
        if st != FEC_OK:
            raise FecError(st, "fec_cluster_batch")
        return labels, ks[:nb]

    def submit(self, xyz, d, min_size, max_size, labels_out, deadline_us=0):
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        st, t = fec_serve_submit_deadline(self.handle, xyz.ctypes.data, xyz.size // 3, d, min_size,
                                          max_size, labels_out.ctypes.data, deadline_us)
        if st != FEC_OK:
            raise FecError(st, "fec_serve_submit")
        return t

    def poll(self, ticket, timeout_ms=-1):
        """(status, k).  Status FEC_OK, NOT_READY while queued or running, or
        a final error (TIMEOUT: the request's deadline passed first)."""
        return fec_serve_poll(self.handle, ticket, timeout_ms)

    def serve_stats(self) -> dict:
        return fec_serve_get_stats(self.handle)

    def poll_timed(self, ticket, timeout_ms=-1):
        """(status, k, done_ns): done_ns = CLOCK_MONOTONIC completion time."""
        return fec_serve_poll_timed(self.handle, ticket, timeout_ms)

    def stats(self) -> dict:
        return fec_get_stats(self.handle)

    def trace(self, enable: bool = True):
        st = fec_trace_enable(self.handle, enable)
        if st != FEC_OK:
            raise FecError(st, "fec_trace_enable")

    def trace_read(self) -> list:
        return fec_trace_read(self.handle)

    def set_iteration_caps(self, wait_cap=FEC_DEFAULT_WAIT_CAP, union_cap=FEC_DEFAULT_UNION_CAP):
        st = fec_set_iteration_caps(self.handle, wait_cap, union_cap)
        if st != FEC_OK:
            raise FecError(st, "fec_set_iteration_caps")
