"""Argument checks of every C ABI entry point, which come before any CUDA call,
so they run here without a GPU: a null context, bad sizes, radii and bounds
are refused with FEC_ERR_INVALID_ARG and nothing is written."""
import ctypes
import math

import numpy as np
import pytest

from paper_2208_07678_gb300 import build as libbuild
from paper_2208_07678_gb300 import fec

OK, INVALID = 0, 1
I64MAX = (1 << 63) - 1


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return fec.load()


def _f32(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def test_null_context_is_refused_everywhere(lib):
    xyz = np.zeros((4, 3), np.float32)
    labels = np.zeros(4, np.int32)
    k = ctypes.c_int32(-7)
    assert lib.fec_cluster(None, _f32(xyz), 4, 0.5, 1, I64MAX, _f32(labels), ctypes.byref(k)) == INVALID
    offs = np.array([0, 4], np.int64)
    d = np.array([0.5], np.float32)
    mn = np.array([1], np.int64)
    mx = np.array([I64MAX], np.int64)
    ks = np.zeros(1, np.int32)
    assert lib.fec_cluster_batch(None, _f32(xyz), _f32(offs), 1, _f32(d), _f32(mn), _f32(mx),
                                 _f32(labels), _f32(ks)) == INVALID
    t = ctypes.c_uint64(0)
    assert lib.fec_serve_submit(None, _f32(xyz), 4, 0.5, 1, I64MAX, _f32(labels), ctypes.byref(t)) == INVALID
    assert lib.fec_serve_poll(None, 1, ctypes.byref(k), 0) == INVALID
    assert lib.fec_serve_poll_timed(None, 1, ctypes.byref(k), 0, None) == INVALID
    assert lib.fec_trace_enable(None, 1) == INVALID
    assert lib.fec_trace_read(None, None, 0) == -1
    assert lib.fec_get_stats(None, ctypes.byref(fec.fec_stats())) == INVALID
    lib.fec_destroy(None)  # a no-op
    assert k.value == -7 and not labels.any()


@pytest.mark.parametrize("n,d,mn,mx", [
    (-1, 0.5, 1, I64MAX),          # negative size
    (40_000, 0.5, 1, I64MAX),      # above the no-allocation entry point's 32,768 points
    (10, 0.0, 1, I64MAX),          # d must be > 0
    (10, -0.5, 1, I64MAX),
    (10, math.nan, 1, I64MAX),
    (10, math.inf, 1, I64MAX),
    (10, 0.5, -1, I64MAX),         # bounds: 0 <= min <= max
    (10, 0.5, 5, 4),
])
def test_noalloc_argument_checks(lib, n, d, mn, mx):
    xyz = np.zeros((max(n, 1), 3), np.float32)
    labels = np.full(max(n, 1), -9, np.int32)
    k = ctypes.c_int32(-7)
    st = lib.fec_cluster_noalloc(_f32(xyz), n, d, mn, mx, _f32(labels), ctypes.byref(k), None)
    assert st == INVALID
    assert np.all(labels == -9)


def test_noalloc_null_buffers_and_empty_cloud(lib):
    k = ctypes.c_int32(-7)
    labels = np.zeros(3, np.int32)
    assert lib.fec_cluster_noalloc(None, 3, 0.5, 1, I64MAX, _f32(labels), ctypes.byref(k), None) == INVALID
    xyz = np.zeros((3, 3), np.float32)
    assert lib.fec_cluster_noalloc(_f32(xyz), 3, 0.5, 1, I64MAX, None, ctypes.byref(k), None) == INVALID
    assert lib.fec_cluster_noalloc(_f32(xyz), 3, 0.5, 1, I64MAX, _f32(labels), None, None) == INVALID
    # n = 0 needs no device: OK with no clusters
    assert lib.fec_cluster_noalloc(None, 0, 0.5, 1, I64MAX, None, ctypes.byref(k), None) == OK
    assert k.value == 0
