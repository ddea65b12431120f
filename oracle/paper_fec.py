"""Algorithm 1 (FEC's serial point-wise loop) as printed, for comparison only.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Algorithm 1 visits the points in index order.  A still-unlabelled point p_i
queries its neighbours within d, takes the smallest non-zero neighbour label
(or a fresh segment label), and rewrites every larger neighbour label across
the whole cloud (the segment-merge loop).  As printed, the loop never writes
the chosen label into p_i or into unlabelled neighbours; this restatement
reads it as doing so (otherwise no point is ever labelled).

Because only still-unlabelled points issue queries, an edge between two points
that were both labelled by earlier queries is never examined.  The result can
therefore split a connected component, which is why the library computes exact
connected components instead (the oracle in ``fec_oracle.c``).  The tests use
this routine to demonstrate that difference on a four-point example.

``paper_fec_serial`` is pure Python, O(n) per query: tiny inputs only.
``paper_fec_serial_kd`` runs the same loop with FindNeighbor answered by a
kd-tree (scipy), for clouds of tens of thousands of points, and
``compare_with_exact`` reports how its size-filtered segments differ from the
exact components.
"""
from __future__ import annotations

import math

import numpy as np


def paper_fec_serial(q: np.ndarray, T2: int) -> np.ndarray:
    """Labels (1-based segment labels, Algorithm 1) from int coordinates q[n,3]."""
    q = np.asarray(q, dtype=np.int64).reshape(-1, 3)
    n = q.shape[0]
    lab = np.zeros(n, dtype=np.int64)
    seg = 1
    for i in range(n):
        if lab[i] != 0:
            continue
        d2 = ((q - q[i]) ** 2).sum(axis=1)
        nn = np.nonzero(d2 <= T2)[0]  # FindNeighbor(p_i, d), p_i included
        nonzero = [lab[j] for j in nn if lab[j] != 0]
        m = min(nonzero + [seg]) if nonzero else seg
        for j in nn:
            old = lab[j]
            if old > m:  # segment merge: rewrite that label everywhere
                lab[lab == old] = m
            elif old == 0:
                lab[j] = m
        seg += 1
    return lab


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
    lab = np.zeros(n, dtype=np.int64)
    if n == 0:
        return lab
    tree = cKDTree(q.astype(np.float64))
    r = math.sqrt(float(T2)) + 1.0
    seg = 1
    for i in range(n):
        if lab[i] != 0:
            continue
        cand = np.sort(np.asarray(tree.query_ball_point(q[i].astype(np.float64), r), dtype=np.int64))
        d2 = ((q[cand] - q[i]) ** 2).sum(axis=1)
        nn = cand[d2 <= T2]
        old = np.unique(lab[nn])
        old = old[old != 0]
        m = int(min(old.min(), seg)) if old.size else seg
        for o in old[old > m]:  # segment merge: rewrite that label everywhere
            lab[lab == o] = m
        lab[nn[lab[nn] == 0]] = m
        seg += 1
    return lab


def compare_with_exact(xyz, d: float, min_size: int = 1, max_size: int = (1 << 63) - 1) -> dict:
    """Algorithm 1 as printed (serial, index order) against the exact
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
