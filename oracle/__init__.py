"""CPU oracle for exact Euclidean clustering (FEC).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA product path never imports it, and it shares no code with
the CUDA path.

What it computes is the plain definition (Eq. 1 and Algorithm 1's input and
output, Section 2.2): the connected components of the graph that joins two
points when their distance is at most ``d``, after quantising coordinates to
1/1024 m with round-half-to-even; components outside ``[min_size, max_size]``
get label -1 (the EC size bounds of Section 3.1); kept components are numbered
0..k-1 by their smallest point index.

The C file ``fec_oracle.c`` is compiled with gcc on first use (or by
``build()``), in-tree, next to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fec_oracle.c")
_LIB = os.path.join(_HERE, "_fec_oracle.so")

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NONFINITE", 3: "OUT_OF_RANGE", 4: "OOM"}

INT64_MAX = (1 << 63) - 1

_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int):
        self.code = code
        self.name = STATUS_NAMES.get(code, f"UNKNOWN({code})")
        super().__init__(f"oracle status {self.name}")


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C, -O2, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        f32p = ctypes.POINTER(ctypes.c_float)
        i32p = ctypes.POINTER(ctypes.c_int32)
        for name in ("fec_oracle_cluster", "fec_oracle_bruteforce"):
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [f32p, ctypes.c_int64, ctypes.c_float, ctypes.c_int64,
                           ctypes.c_int64, i32p, i32p]
        lib.fec_oracle_quantize.restype = ctypes.c_int
        lib.fec_oracle_quantize.argtypes = [f32p, ctypes.c_int64, i32p]
        lib.fec_oracle_threshold.restype = ctypes.c_int64
        lib.fec_oracle_threshold.argtypes = [ctypes.c_float]
        lib.fec_oracle_components.restype = ctypes.c_int
        lib.fec_oracle_components.argtypes = [i32p, ctypes.c_int64, ctypes.c_int64, i32p]
        _lib = lib
    return _lib


def _as_xyz(xyz) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32))
    if a.ndim != 2 or a.shape[1] != 3:
        a = a.reshape(-1, 3)
    return a


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _cluster(fn_name, xyz, d, min_size, max_size):
    lib = _load()
    a = _as_xyz(xyz)
    n = a.shape[0]
    labels = np.empty(max(n, 1), dtype=np.int32)
    k = ctypes.c_int32(-7)
    st = getattr(lib, fn_name)(_ptr(a, ctypes.c_float), n, float(d), int(min_size),
                               int(max_size), _ptr(labels, ctypes.c_int32), ctypes.byref(k))
    if st != 0:
        raise OracleError(st)
    return labels[:n], int(k.value)


def cluster(xyz, d: float, min_size: int = 1, max_size: int = INT64_MAX):
    """kd-tree BFS oracle.  Returns (labels int32[n], k).  Raises OracleError."""
    return _cluster("fec_oracle_cluster", xyz, d, min_size, max_size)


def _cluster_job(job):
    xyz, d, min_size, max_size = job
    return cluster(xyz, d, min_size, max_size)


def cluster_many(jobs, processes=None):
    """cluster() over independent clouds [(xyz, d, min_size, max_size), ...]
    in a pool of worker processes (one per host core by default), in order.
    The pool is started with ``spawn``, so it is safe in a process that
    already uses the GPU.  Returns [(labels, k), ...]."""
    import multiprocessing as mp

    jobs = list(jobs)
    if not jobs:
        return []
    procs = processes or os.cpu_count() or 1
    procs = max(1, min(procs, len(jobs)))
    if procs == 1:
        return [_cluster_job(j) for j in jobs]
    build()  # compile once here, not in every worker
    # largest clouds first, so that no worker is left with a big one at the end
    order = sorted(range(len(jobs)), key=lambda i: -np.asarray(jobs[i][0]).size)
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_cluster_job, [jobs[i] for i in order], chunksize=1)
    out = [None] * len(jobs)
    for i, r in zip(order, res):
        out[i] = r
    return out


def bruteforce(xyz, d: float, min_size: int = 1, max_size: int = INT64_MAX):
    """O(n^2) all-pairs union-find oracle (tiny inputs only)."""
    return _cluster("fec_oracle_bruteforce", xyz, d, min_size, max_size)


def status_of(fn, *args, **kw) -> str:
    """Run an oracle call and return its status name ('OK' on success)."""
    try:
        fn(*args, **kw)
        return "OK"
    except OracleError as e:
        return e.name


def quantize(xyz) -> np.ndarray:
    """q = rint(x * 1024) as int32[n, 3] (round half to even)."""
    lib = _load()
    a = _as_xyz(xyz)
    q = np.zeros(a.shape, dtype=np.int32)
    st = lib.fec_oracle_quantize(_ptr(a, ctypes.c_float), a.shape[0], _ptr(q, ctypes.c_int32))
    if st != 0:
        raise OracleError(st)
    return q


def threshold(d: float) -> int:
    """T2 = floor((d * 1024)^2), the squared join radius in integer units."""
    return int(_load().fec_oracle_threshold(float(d)))


def components(q, T2: int) -> np.ndarray:
    """comp[i] = smallest index of i's component, from int32 coordinates."""
    lib = _load()
    qa = np.ascontiguousarray(np.asarray(q, dtype=np.int32).reshape(-1, 3))
    comp = np.empty(max(qa.shape[0], 1), dtype=np.int32)
    st = lib.fec_oracle_components(_ptr(qa, ctypes.c_int32), qa.shape[0], int(T2),
                                   _ptr(comp, ctypes.c_int32))
    if st != 0:
        raise OracleError(st)
    return comp[: qa.shape[0]]


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)
