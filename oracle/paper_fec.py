"""FEC's serial point-wise scheme, for comparison with the exact components.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 2 describes FEC as a point-wise scheme: points are visited in their
input order, and only a point that no earlier visit has put into a segment
looks for its neighbours within d (FindNeighbor, Algorithm 1).  The segments
already present around it are merged into the one with the smallest segment
number (a fresh number when there is none), and the neighbours that had no
segment join it.  The printed listing leaves the chosen number unwritten for
the visiting point and its unlabelled neighbours; this module reads it as
writing it (otherwise no point would ever be labelled).

Here the scheme is kept as a partition of segment numbers (a small
union-find whose root is the smallest number of each merged group) instead of
relabelling the whole cloud at every merge; the partition it yields is the
same.  Because only points without a segment issue queries, an edge between
two points that earlier visits both put into segments is never examined: the
result can split a connected component of the distance graph, which is why
the library computes exact components (the oracle in ``fec_oracle.c``).

``paper_fec_serial`` answers each neighbour query by brute force (tiny
inputs only); ``paper_fec_serial_kd`` by a kd-tree (scipy), for clouds of
tens of thousands of points; ``compare_with_exact`` reports how the
size-filtered segments differ from the exact components.
"""
from __future__ import annotations

import math

import numpy as np


class _Segments:
    """Segment numbers 1, 2, ... under merging; the representative of a
    merged group is its smallest number."""

    def __init__(self):
        self.up = [0]  # up[s] == s for a representative; slot 0 is unused

    def new(self) -> int:
        self.up.append(len(self.up))
        return len(self.up) - 1

    def rep(self, s: int) -> int:
        while self.up[s] != s:
            self.up[s] = self.up[self.up[s]]
            s = self.up[s]
        return s

    def merge_into(self, keep: int, others) -> None:
        for o in others:
            self.up[self.rep(o)] = keep


def _pointwise(n: int, neighbours) -> np.ndarray:
    """The point-wise scheme over points 0..n-1; neighbours(i) returns the
    indices within d of point i (i included).  Returns 1-based labels."""
    seg = np.zeros(n, dtype=np.int64)  # 0: no segment yet
    segs = _Segments()
    for i in range(n):
        if seg[i]:
            continue
        near = neighbours(i)
        fresh = segs.new()
        present = {segs.rep(int(s)) for s in seg[near] if s}
        keep = min(present | {fresh})
        segs.merge_into(keep, present | {fresh})
        free = near[seg[near] == 0]
        seg[free] = keep
    return np.array([segs.rep(int(s)) for s in seg], dtype=np.int64)


def paper_fec_serial(q: np.ndarray, T2: int) -> np.ndarray:
    """Segment labels of the point-wise scheme from int coordinates q[n,3],
    neighbours by brute force (join iff squared distance <= T2)."""
    q = np.asarray(q, dtype=np.int64).reshape(-1, 3)

    def neighbours(i):
        return np.nonzero(((q - q[i]) ** 2).sum(axis=1) <= T2)[0]

    return _pointwise(q.shape[0], neighbours)


def canonical(labels: np.ndarray) -> np.ndarray:
    """Renumber a partition 0..k-1 by the smallest index of each part."""
    labels = np.asarray(labels)
    out = np.empty(labels.shape[0], dtype=np.int32)
    seen: dict = {}
    for i, v in enumerate(labels.tolist()):
        if v not in seen:
            seen[v] = len(seen)
        out[i] = seen[v]
    return out


def paper_fec_serial_kd(q: np.ndarray, T2: int) -> np.ndarray:
    """paper_fec_serial with the neighbour query through a kd-tree: the same
    labels, for larger clouds (candidates within sqrt(T2) + 1 units, then the
    exact integer test)."""
    from scipy.spatial import cKDTree

    q = np.asarray(q, dtype=np.int64).reshape(-1, 3)
    n = q.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    tree = cKDTree(q.astype(np.float64))
    r = math.sqrt(float(T2)) + 1.0

    def neighbours(i):
        cand = np.asarray(tree.query_ball_point(q[i].astype(np.float64), r), dtype=np.int64)
        return cand[((q[cand] - q[i]) ** 2).sum(axis=1) <= T2]

    return _pointwise(n, neighbours)


def compare_with_exact(xyz, d: float, min_size: int = 1, max_size: int = (1 << 63) - 1) -> dict:
    """The point-wise scheme (serial, index order) against the exact
    components on one cloud, both with the size bounds applied: cluster
    counts, exact components that the serial loop splits, and the points
    whose kept/dropped state or partner set differs."""
    from . import cluster, components, quantize, threshold

    q = quantize(xyz)
    T2 = threshold(d)
    exact_lab, k_exact = cluster(xyz, d, min_size, max_size)
    comp = components(q, T2)
    seg = paper_fec_serial_kd(q, T2)
    # serial segments, size-filtered like the exact ones
    _, seg_id, seg_size = np.unique(seg, return_inverse=True, return_counts=True)
    seg_kept = (seg_size[seg_id] >= min_size) & (seg_size[seg_id] <= max_size)
    k_serial = int(np.unique(seg_id[seg_kept]).size)
    # every serial segment lies inside one exact component (it only grows
    # along edges); an exact component is split when it holds several segments
    pairs = np.unique(np.stack([comp, seg_id], axis=1), axis=0)
    per_comp = np.bincount(pairs[:, 0], minlength=len(q))
    split_comps = int(np.count_nonzero(per_comp > 1))
    in_split = per_comp[comp] > 1
    same_state = (exact_lab >= 0) == seg_kept
    return {"n": int(len(q)), "k_exact": int(k_exact), "k_serial": k_serial,
            "components_split": split_comps, "points_in_split_components": int(in_split.sum()),
            "points_kept_state_differs": int(np.count_nonzero(~same_state))}
