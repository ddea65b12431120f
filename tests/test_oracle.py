"""Pins for the CPU oracle, checked against things other than itself:
hand-derived fixtures (tests/golden), closed forms, invariants, brute force,
an independent scipy route, and generator ground truth (Section 3.3.1)."""
import numpy as np
import pytest

import oracle
from oracle.paper_fec import canonical, compare_with_exact, paper_fec_serial, paper_fec_serial_kd
from paper_2208_07678_gb300 import synth
from tests._util import (INT64_MAX, boundary_pairs, check_labels_valid, fixtures, quantize_np,
                         random_cloud, scipy_labels, threshold_np)

FIXTURES = fixtures()


@pytest.mark.parametrize("fx", FIXTURES, ids=[f["name"] for f in FIXTURES])
def test_golden_fixture_kdtree(fx):
    lab, k = oracle.cluster(fx["xyz"], fx["d"], fx["min_size"], fx["max_size"])
    assert k == fx["k"], fx["cite"]
    np.testing.assert_array_equal(lab, fx["labels"], err_msg=fx["cite"])


@pytest.mark.parametrize("fx", FIXTURES, ids=[f["name"] for f in FIXTURES])
def test_golden_fixture_bruteforce(fx):
    lab, k = oracle.bruteforce(fx["xyz"], fx["d"], fx["min_size"], fx["max_size"])
    assert k == fx["k"]
    np.testing.assert_array_equal(lab, fx["labels"])


def test_quantize_matches_numpy_rint_half_even():
    x = np.array([[0.5 / 1024, 1.5 / 1024, 2.5 / 1024],
                  [-0.5 / 1024, -1.5 / 1024, -2.5 / 1024],
                  [1234.5678, -0.0001, 8191.999]], dtype=np.float32)
    q = oracle.quantize(x)
    np.testing.assert_array_equal(q[0], [0, 2, 2])
    np.testing.assert_array_equal(q[1], [0, -2, -2])
    np.testing.assert_array_equal(q, quantize_np(x))
    rng = np.random.default_rng(11)
    y = rng.uniform(-8000, 8000, size=(5000, 3)).astype(np.float32)
    np.testing.assert_array_equal(oracle.quantize(y), quantize_np(y))


def test_quantize_errors_and_precedence():
    ok = np.zeros((3, 3), np.float32)
    for bad, want in [(np.nan, "NONFINITE"), (np.inf, "NONFINITE"), (-np.inf, "NONFINITE"),
                      (8192.0, "OUT_OF_RANGE"), (-8192.0, "OUT_OF_RANGE"),
                      (8191.9995, "OUT_OF_RANGE")]:
        x = ok.copy()
        x[1, 2] = bad
        assert oracle.status_of(oracle.cluster, x, 0.5) == want, (bad, want)
    x = ok.copy()
    x[0, 0] = 8192.0
    x[2, 1] = np.nan
    assert oracle.status_of(oracle.cluster, x, 0.5) == "NONFINITE"
    x = ok.copy()
    x[0, 0] = 8191.999
    assert oracle.status_of(oracle.cluster, x, 0.5) == "OK"  # rint -> 2^23 - 1


def test_argument_errors():
    x = np.zeros((4, 3), np.float32)
    for d in (0.0, -1.0, float("nan"), float("inf")):
        assert oracle.status_of(oracle.cluster, x, d) == "INVALID_ARG"
    assert oracle.status_of(oracle.cluster, x, 0.5, 3, 2) == "INVALID_ARG"
    assert oracle.status_of(oracle.cluster, x, 0.5, -1, 2) == "INVALID_ARG"
    assert oracle.status_of(oracle.cluster, x, 0.5, 0, 0) == "OK"


@pytest.mark.parametrize("d", [0.5, 0.2, 0.35, 1.0 / 1024, 0.1234, 7.0, 1e-9])
def test_threshold_closed_form(d):
    assert oracle.threshold(d) == threshold_np(d)


def test_threshold_pins():
    assert oracle.threshold(0.5) == 512 * 512
    assert oracle.threshold(0.2) == 41943  # floor(204.80000305^2)
    assert oracle.threshold(1e30) == 1 << 62  # capped


@pytest.mark.parametrize("seed", range(12))
def test_kdtree_equals_bruteforce_and_scipy(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 1500))
    xyz = random_cloud(seed, n, extent=float(rng.uniform(1, 6)), clumps=int(rng.integers(0, 8)))
    d = float(np.float32(rng.choice([0.05, 0.1, 0.2, 0.3, 0.5, 0.75])))
    mn = int(rng.integers(0, 4))
    mx = int(rng.choice([INT64_MAX, 5, 40, 400]))
    a = oracle.cluster(xyz, d, mn, mx)
    b = oracle.bruteforce(xyz, d, mn, mx)
    c = scipy_labels(xyz, d, mn, mx)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[0], c[0])
    assert a[1] == b[1] == c[1]


def test_components_seed_is_smallest_index():
    xyz = random_cloud(5, 800, extent=3.0, clumps=5)
    q = oracle.quantize(xyz)
    comp = oracle.components(q, oracle.threshold(0.2))
    for c in np.unique(comp):
        assert np.nonzero(comp == c)[0].min() == c


@pytest.mark.parametrize("seed", range(4))
def test_permutation_invariance(seed):
    """The paper shuffles the point index (Section 3.3.1); the partition must
    not depend on it.  Renumbering by smallest index restores equality."""
    xyz = random_cloud(seed, 3000, extent=5.0, clumps=10)
    lab, k = oracle.cluster(xyz, 0.2, 2, 300)
    perm = np.random.default_rng(seed).permutation(len(xyz))
    lab_p, k_p = oracle.cluster(xyz[perm], 0.2, 2, 300)
    assert k == k_p
    # lab_p[j] is the label of original point perm[j]; compare partitions.
    back = np.empty_like(lab_p)
    back[perm] = lab_p
    kept = lab >= 0
    np.testing.assert_array_equal(kept, back >= 0)
    np.testing.assert_array_equal(canonical(lab[kept]), canonical(back[kept]))


@pytest.mark.parametrize("shift_units", [(1, 0, 0), (37, -511, 1023), (-4096, 4096, 12345)])
def test_translation_by_grid_multiples(shift_units):
    xyz = random_cloud(9, 2500, extent=4.0, clumps=6)
    shift = np.asarray(shift_units, dtype=np.float64) / 1024.0
    moved = (xyz.astype(np.float64) + shift).astype(np.float32)
    a = oracle.cluster(xyz, 0.25, 1, 500)
    b = oracle.cluster(moved, 0.25, 1, 500)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1] == b[1]


@pytest.mark.parametrize("seed", range(3))
def test_output_properties(seed):
    xyz = random_cloud(seed, 4000, extent=6.0, clumps=12)
    lab, k = oracle.cluster(xyz, 0.15, 3, 200)
    check_labels_valid(xyz, 0.15, lab, k, 3, 200)


def test_kept_clusters_are_connected():
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    from tests._util import scipy_edges

    xyz = random_cloud(3, 2000, extent=4.0, clumps=8)
    lab, k = oracle.cluster(xyz, 0.2)
    q = quantize_np(xyz)
    for c in range(min(k, 30)):
        idx = np.nonzero(lab == c)[0]
        e = scipy_edges(q[idx], threshold_np(0.2))
        g = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(len(idx), len(idx)))
        assert connected_components(g, directed=False)[0] == 1


@pytest.mark.parametrize("n_clusters,density,d", [(40, 27, 0.4), (100, 64, 0.3), (25, 200, 0.2)])
def test_voxel_generator_ground_truth(n_clusters, density, d):
    """Section 3.3.1 recipe: m points evenly filled into n separated voxels.
    With lattice spacing <= d < gap, the answer is n clusters of m points."""
    xyz = synth.voxel_clusters(seed=7, n_clusters=n_clusters, density=density)
    lab, k = oracle.cluster(xyz, d)
    assert k == n_clusters
    assert np.all(np.bincount(lab) == density)


def test_fig3_extremes_on_random_cloud():
    """Fig. 3: maximum d gives one cluster, minimum d gives singletons."""
    rng = np.random.default_rng(4)
    pts = rng.choice(200 ** 3, size=500, replace=False)
    xyz = (np.stack([pts % 200, (pts // 200) % 200, pts // 40000], 1) * 3 / 1024).astype(np.float32)
    lab, k = oracle.cluster(xyz, 1000.0)
    assert k == 1 and np.all(lab == 0)
    lab, k = oracle.cluster(xyz, 2.0 / 1024)  # distinct points are >= 3 units apart
    assert k == 500
    np.testing.assert_array_equal(lab, np.arange(500))


def test_serial_algorithm_differs_from_exact_components():
    """Algorithm 1's point-wise loop (as printed) splits a chain that exact
    connected components (Eq. 1) keep whole."""
    q = np.array([[0, 0, 0], [3, 0, 0], [1, 0, 0], [2, 0, 0]]) * 1024
    serial = canonical(paper_fec_serial(q, 1024 * 1024))
    np.testing.assert_array_equal(serial, [0, 1, 0, 1])
    lab, k = oracle.cluster(q.astype(np.float32) / 1024, 1.0)
    assert k == 1 and np.all(lab == 0)


def test_serial_algorithm_agrees_when_order_is_spatial():
    """On a chain visited in spatial order Algorithm 1 and the exact
    components agree (sanity check of the serial restatement)."""
    q = np.array([[i, 0, 0] for i in range(6)]) * 1024
    q = np.concatenate([q, q + [100 * 1024, 0, 0]])
    serial = canonical(paper_fec_serial(q, 1024 * 1024))
    lab, _ = oracle.cluster(q.astype(np.float32) / 1024, 1.0)
    np.testing.assert_array_equal(serial, lab)


def test_planted_mistake_is_caught():
    """A wrong join rule (strict < d instead of <= d) fails the equality
    fixture: the pins can tell the two readings apart."""
    fx = [f for f in FIXTURES if f["name"] == "pair_exact_d.txt"][0]
    q = quantize_np(fx["xyz"])
    T2 = threshold_np(fx["d"])
    strict = ((q[0] - q[1]) ** 2).sum() < T2
    assert not strict  # the strict reading would split the pair
    lab, k = oracle.cluster(fx["xyz"], fx["d"])
    assert k == 1


@pytest.mark.parametrize("d", [0.05, 0.35, 3.0])
def test_pairs_at_the_threshold(d):
    """Closed form: isolated pairs (5d apart) join iff their squared distance
    in quantised units is at most T2 = floor((d*1024)^2) (Eq. 1 with the
    quantisation reading); pairs sit within a few units of T2 on both sides,
    including axis-aligned pairs at exactly R and R + 1."""
    xyz, joined = boundary_pairs(d, seed=int(d * 1000) + 1)
    labels, k = oracle.cluster(xyz, d, 1, INT64_MAX)
    m = len(joined)
    assert k == int(joined.sum()) + 2 * int((~joined).sum())
    np.testing.assert_array_equal(labels[:m] == labels[m:], joined)



@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_serial_kd_loop_equals_plain_loop(seed):
    """The kd-tree FindNeighbor gives the same Algorithm 1 labels as the
    all-points scan."""
    rng = np.random.default_rng([seed, 31])
    n = int(rng.integers(1, 400))
    q = rng.integers(-3000, 3000, size=(n, 3))
    T2 = int(rng.integers(1, 400_000))
    np.testing.assert_array_equal(canonical(paper_fec_serial(q, T2)),
                                  canonical(paper_fec_serial_kd(q, T2)))


def test_serial_segments_refine_exact_components():
    """Algorithm 1 only merges along edges, so each of its segments lies in
    one exact component; it may split a component, never join two."""
    xyz = random_cloud(5, 3000, extent=10.0, clumps=12)
    q, T2 = oracle.quantize(xyz), oracle.threshold(0.3)
    comp = oracle.components(q, T2)
    seg = paper_fec_serial_kd(q, T2)
    for s in np.unique(seg):
        assert np.unique(comp[seg == s]).size == 1
    assert np.unique(seg).size >= np.unique(comp).size


def test_serial_report_on_the_counterexample():
    xyz = np.array([[0, 0, 0], [3, 0, 0], [1, 0, 0], [2, 0, 0]], dtype=np.float32)
    r = compare_with_exact(xyz, 1.0)
    assert (r["k_exact"], r["k_serial"], r["components_split"], r["points_in_split_components"]) == (1, 2, 1, 4)
    assert r["points_kept_state_differs"] == 0
