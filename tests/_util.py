"""Helpers shared by the tests: fixture parsing and independent checks.

The independent checks here use scipy (cKDTree pairs + connected components),
a route that shares nothing with the oracle's kd-tree BFS or with the CUDA
library.
"""
from __future__ import annotations

import glob
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INT64_MAX = (1 << 63) - 1


def load_fixture(path):
    d = mn = mx = None
    pts, labels, k, cite = [], None, None, []
    mode = None
    with open(path) as f:
        for raw in f:
            line = raw.strip()
            if line.startswith("#"):
                cite.append(line[1:].strip())
                continue
            if mode == "points" and line and line != "labels":
                pts.append([float(v) for v in line.split()])
                continue
            if mode == "labels_next":
                labels = [int(v) for v in line.split()]
                mode = None
                continue
            if not line:
                continue
            key, *rest = line.split()
            if key == "d":
                d = float(rest[0])
            elif key == "min":
                mn = int(rest[0])
            elif key == "max":
                mx = INT64_MAX if rest[0] == "inf" else int(rest[0])
            elif key == "points":
                mode = "points"
            elif key == "labels":
                mode = "labels_next"
            elif key == "k":
                k = int(rest[0])
    xyz = np.asarray(pts, dtype=np.float32).reshape(-1, 3)
    return dict(name=os.path.basename(path), cite=" ".join(cite), xyz=xyz, d=d, min_size=mn,
                max_size=mx, labels=np.asarray(labels or [], dtype=np.int32), k=k)


def fixtures():
    return [load_fixture(p) for p in sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))
            if not p.endswith("README.txt")]


def quantize_np(xyz):
    """Independent quantisation: numpy rint (half to even) of float32 * 1024."""
    return np.rint(np.asarray(xyz, dtype=np.float32) * np.float32(1024)).astype(np.int64)


def threshold_np(d):
    s = float(np.float32(d)) * 1024.0
    return int(np.floor(s * s))


def scipy_edges(q, T2):
    """All pairs with integer squared distance <= T2 (scipy kd-tree + exact filter)."""
    from scipy.spatial import cKDTree

    q = np.asarray(q, dtype=np.int64)
    if q.shape[0] < 2:
        return np.zeros((0, 2), dtype=np.int64)
    tree = cKDTree(q.astype(np.float64))
    pairs = tree.query_pairs(np.sqrt(T2) + 1e-6, output_type="ndarray")
    if pairs.size == 0:
        return pairs.reshape(0, 2)
    dd = ((q[pairs[:, 0]] - q[pairs[:, 1]]) ** 2).sum(axis=1)
    return pairs[dd <= T2]


def scipy_labels(xyz, d, min_size=1, max_size=INT64_MAX):
    """Reference labels computed with scipy's graph routines."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    q = quantize_np(xyz)
    n = q.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.int32), 0
    e = scipy_edges(q, threshold_np(d))
    g = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    return canonical_filter(comp, min_size, max_size)


def canonical_filter(comp, min_size=1, max_size=INT64_MAX):
    """Partition -> labels: filter by size, number kept parts by smallest index."""
    comp = np.asarray(comp)
    n = comp.shape[0]
    uniq, first, counts = np.unique(comp, return_index=True, return_counts=True)
    keep = (counts >= min_size) & (counts <= max_size)
    order = np.argsort(first[keep], kind="stable")
    number = np.full(uniq.shape[0], -1, dtype=np.int64)
    kept_idx = np.nonzero(keep)[0][order]
    number[kept_idx] = np.arange(kept_idx.shape[0])
    lab = number[np.searchsorted(uniq, comp)]
    return lab.astype(np.int32), int(kept_idx.shape[0])


def check_labels_valid(xyz, d, labels, k, min_size=1, max_size=INT64_MAX):
    """Properties that hold for any correct output, at any size:
    closure (edges never cross labels), dense numbering 0..k-1 by smallest
    index, and kept sizes inside the bounds."""
    labels = np.asarray(labels)
    n = labels.shape[0]
    if n == 0:
        assert k == 0
        return
    kept = labels[labels >= 0]
    if kept.size:
        assert kept.max() == k - 1
        firsts = np.unique(kept, return_index=True)[1]
        idx = np.nonzero(labels >= 0)[0][firsts]
        assert np.all(np.diff(idx) > 0), "kept clusters not numbered by smallest index"
        sizes = np.bincount(kept, minlength=k)
        assert sizes.min() >= min_size and sizes.max() <= max_size
    else:
        assert k == 0
    e = scipy_edges(quantize_np(xyz), threshold_np(d))
    if len(e):
        a, b = labels[e[:, 0]], labels[e[:, 1]]
        assert np.all(a == b), "an edge of length <= d crosses two labels"


def random_cloud(seed, n, extent=4.0, clumps=0):
    rng = np.random.default_rng(seed)
    if clumps:
        c = rng.uniform(0, extent, size=(clumps, 3))
        pts = c[rng.integers(0, clumps, n)] + rng.normal(0, extent / 20, size=(n, 3))
    else:
        pts = rng.uniform(0, extent, size=(n, 3))
    return (np.rint(pts * 1024) / 1024).astype(np.float32)


def boundary_pairs(d, seed):
    """Isolated point pairs at squared distances within a few units of T2
    (both sides), with random alignment to the cell and sub-cell grid, plus
    axis-aligned pairs at exactly R and R+1 in all six directions.  Pairs sit
    5d apart, so only the two points of a pair can join."""
    rng = np.random.default_rng(seed)
    T2 = threshold_np(d)
    R = int(np.floor(np.sqrt(T2)))
    while R * R > T2:
        R -= 1
    while (R + 1) * (R + 1) <= T2:
        R += 1
    step = int(5 * d * 1024)
    g = np.arange(24)
    centres = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * step
    centres += rng.integers(0, max(1, step // 5), size=centres.shape)
    m = len(centres)
    u = rng.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    length = np.sqrt(T2) + rng.uniform(-1.5, 1.5, size=(m, 1))
    off = np.rint(u * length).astype(np.int64)
    axis = np.zeros((12, 3), np.int64)
    for i in range(6):
        axis[2 * i, i // 2] = (R if i % 2 == 0 else -R)
        axis[2 * i + 1, i // 2] = (R + 1 if i % 2 == 0 else -(R + 1))
    off[: len(axis)] = axis
    q = np.concatenate([centres, centres + off])
    xyz = (q / 1024.0).astype(np.float32)
    joined = (off * off).sum(1) <= T2
    return xyz, joined

