"""The grid geometry the CUDA path relies on, checked on the CPU from its
definition (no code shared with the kernels): with T2 = floor((d*1024)^2),
R = isqrt(T2), h = max(1, ceil(R/2)) and cells of side S = 2h,

* every joined pair lies in the same or an adjacent cell (S >= R);
* a sub-cell (side h) is a clique: 3 (h-1)^2 <= T2;
* the static sub-cell-code filter is exact: along an axis where the neighbour
  cell is at +1, a point in the lower half of its cell and one in the upper
  half of the next cell are at least 2h + 1 > R apart;
* the multiply-shift division floor(rel / S) == (rel * m) >> s, with
  s = 24 + ceil(log2 S) and m = ceil(2^s / S), is exact for every rel < 2^24.
"""
import math

import numpy as np
import pytest

import oracle


def grid_of(d):
    T2 = oracle.threshold(d)
    R = math.isqrt(T2)
    h = max(1, (R + 1) // 2)
    return T2, R, h, 2 * h


RADII = sorted({float(v) for v in np.concatenate([
    np.arange(1, 4097) / 1024.0,                      # every radius up to 4 m on the 1/1024 grid
    np.geomspace(1.0 / 4096, 2000.0, 3000),           # and off-grid ones up to 2 km
])})


def test_cells_hold_every_joined_pair_and_sub_cells_are_cliques():
    for d in RADII:
        T2, R, h, S = grid_of(d)
        assert R * R <= T2 < (R + 1) * (R + 1)
        assert S >= R, d                     # adjacent cells suffice (27-cell stencil)
        assert 3 * (h - 1) ** 2 <= T2, d     # a sub-cell is a clique


def test_static_filter_gap_exceeds_the_radius():
    for d in RADII:
        T2, R, h, S = grid_of(d)
        # lower half of cell c (offsets 0..h-1) against upper half of cell c+1
        # (offsets S+h .. 2S-1): the smallest per-axis gap
        gap = (S + h) - (h - 1)
        assert gap == 2 * h + 1 and gap * gap > T2, d


@pytest.mark.parametrize("d", [0.05, 0.2, 0.35, 1.0])
def test_static_filter_on_points(d):
    """Brute force: random points in the filtered sub-cell pairs never join,
    and the pairs the filter keeps do contain joinable points."""
    T2, R, h, S = grid_of(d)
    rng = np.random.default_rng(int(d * 1000))
    lo = rng.integers(0, h, size=(4000, 1))              # lower half of cell 0
    hi = S + h + rng.integers(0, h, size=(4000, 1))      # upper half of cell 1
    other = rng.integers(0, 2 * S, size=(4000, 2)) - S   # any offsets on the other axes
    a = np.concatenate([lo, other[:, :1], other[:, 1:]], axis=1)
    b = np.concatenate([hi, other[::-1, :1], other[::-1, 1:]], axis=1)
    assert np.all(((a - b) ** 2).sum(axis=1) > T2)
    # a kept configuration (upper half of cell 0, lower half of cell 1) can join
    assert ((h + (h - 1)) - (S + 0)) ** 2 <= T2


@pytest.mark.parametrize("S", [2, 4, 6, 18, 204, 410, 1000, 1024, 2046, 4096, 12346, 1 << 20])
def test_multiply_shift_division_is_exact(S):
    lg = 0
    while (1 << lg) < S:
        lg += 1
    s = 24 + lg
    m = ((1 << s) + S - 1) // S
    rel = np.arange(1 << 24, dtype=np.uint64)
    got = (rel * np.uint64(m)) >> np.uint64(s)
    np.testing.assert_array_equal(got, rel // np.uint64(S))


def test_cell_keys_fit_for_one_centimetre_over_eight_kilometres():
    """The documented limit: for d >= 1 cm over an 8 km cube the cell key needs
    at most 61 bits (3 axes of bitlen(extent / S)), plus the 3-bit sub-cell code."""
    ext = 8000 * 1024
    for d in [0.01, 0.0101, 0.015, 0.02, 0.1, 1.0, 10.0]:
        _, _, _, S = grid_of(d)
        assert 3 * (ext // S).bit_length() <= 61, d
