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

Pure Python, O(n^2) per query: tiny inputs only.
"""
from __future__ import annotations

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
