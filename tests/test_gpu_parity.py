"""GPU parity: the CUDA library, called through the C ABI, against the CPU
oracle, element by element.  Labels are integers with a unique correct
answer, so the bar is bit-exact equality (no tolerance)."""
import numpy as np
import pytest

import oracle
from paper_2208_07678_gb300 import fec, synth
from tests._util import INT64_MAX, boundary_pairs, check_labels_valid, fixtures, random_cloud

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2208_07678_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    c = fec.Context(device=0)
    yield c
    c.close()


def run_gpu(ctx, xyz, d, mn=1, mx=INT64_MAX, device=True):
    import torch

    if device:
        t = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float32)).cuda()
        lab, k = ctx.cluster(t, d, mn, mx)
        torch.cuda.synchronize()
        return lab.cpu().numpy(), k
    return ctx.cluster(np.ascontiguousarray(xyz, dtype=np.float32), d, mn, mx)


def assert_parity(ctx, xyz, d, mn=1, mx=INT64_MAX, device=True):
    want, kw = oracle.cluster(xyz, d, mn, mx)
    got, kg = run_gpu(ctx, xyz, d, mn, mx, device)
    assert kg == kw, f"k: gpu {kg} oracle {kw}"
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{bad.size} labels differ, first at {bad[:10]}: gpu {got[bad[:10]]} "
                             f"oracle {want[bad[:10]]}")
    return got, kg


FIX = fixtures()


@pytest.mark.parametrize("fx", FIX, ids=[f["name"] for f in FIX])
@pytest.mark.parametrize("device", [True, False], ids=["device", "host"])
def test_golden_fixtures(ctx, fx, device):
    got, k = run_gpu(ctx, fx["xyz"], fx["d"], fx["min_size"], fx["max_size"], device)
    assert k == fx["k"], fx["cite"]
    np.testing.assert_array_equal(got, fx["labels"], err_msg=fx["cite"])


@pytest.mark.parametrize("seed", range(40))
def test_random_small(ctx, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 30000))
    xyz = random_cloud(seed, n, extent=float(rng.uniform(1, 20)), clumps=int(rng.integers(0, 30)))
    d = float(np.float32(rng.choice([0.03, 0.1, 0.15, 0.2, 0.35, 0.5, 0.77, 1.3])))
    mn = int(rng.integers(0, 5))
    mx = int(rng.choice([INT64_MAX, 10, 100, 5000]))
    assert_parity(ctx, xyz, d, mn, mx, device=bool(seed % 2))


def test_blobs_20k(ctx):
    c = synth.blobs_20k()
    assert_parity(ctx, c.xyz, c.d, c.min_size, c.max_size)


def test_frame_120k(ctx):
    c = synth.frame_120k()
    assert_parity(ctx, c.xyz, c.d, c.min_size, c.max_size)


@pytest.mark.parametrize("seed", [11, 12])
def test_batch_frames_sizes(ctx, seed):
    rng = np.random.default_rng(seed)
    for n in (20_000, 180_000):
        xyz = synth.to_grid(synth.frame_of_size(rng, n))
        for d in (0.25, 0.5):
            assert_parity(ctx, xyz, d, 50, 50_000)


def test_voxel_clusters(ctx):
    for n_c, dens, sigma, d in [(500, 200, 0.0, 0.3), (300, 500, 0.05, 0.2), (1000, 64, 0.1, 0.35)]:
        xyz = synth.voxel_clusters(3, n_c, dens, sigma)
        assert_parity(ctx, xyz, d)


# ---------------------------------------------------------------- adversarial

def test_one_dense_cell(ctx):
    rng = np.random.default_rng(5)
    xyz = synth.to_grid(rng.uniform(0, 0.2, size=(100_000, 3)))
    got, k = assert_parity(ctx, xyz, 0.5)
    assert k == 1


def test_dense_near_miss(ctx):
    """Two dense slabs whose closest points are just over d apart."""
    rng = np.random.default_rng(6)
    a = rng.uniform(0, 0.3, size=(40_000, 3))
    b = rng.uniform(0, 0.3, size=(40_000, 3))
    a[:, 0] = rng.uniform(0, 0.1, 40_000)
    b[:, 0] = rng.uniform(0.3 + 1 / 1024, 0.4, 40_000)
    b[0, 0] = 0.3 + 1 / 1024
    a[0, :] = [0.1, b[0, 1], b[0, 2]]
    xyz = synth.to_grid(np.concatenate([a, b]))
    _, k = assert_parity(ctx, xyz, 0.2)
    assert k == 2


def test_long_chain(ctx):
    n = 1_000_000
    rng = np.random.default_rng(7)
    x = np.arange(n, dtype=np.float64) * 0.125
    xyz = np.stack([x % 4000.0, np.floor(x / 4000.0) * 0.125, np.zeros(n)], 1)
    xyz = synth.to_grid(xyz[rng.permutation(n)])
    _, k = assert_parity(ctx, xyz, 0.125)
    assert k == 1


def test_points_on_cell_faces(ctx):
    """Lattice with spacing exactly d: every edge has length d and many
    points sit on cell boundaries."""
    g = np.arange(0, 40) * 0.25
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(8)
    xyz = synth.to_grid(xyz[rng.permutation(len(xyz))])
    _, k = assert_parity(ctx, xyz, 0.25)
    assert k == 1
    _, k = assert_parity(ctx, xyz, 0.25 - 1 / 1024)
    assert k == len(xyz)


def test_range_limits(ctx):
    lim = 8191.99
    xyz = np.array([[lim, 0, 0], [lim - 0.2, 0, 0], [-lim, -lim, -lim], [-lim + 0.1, -lim, -lim],
                    [0, lim, -lim], [0, 0, 0]], dtype=np.float32)
    assert_parity(ctx, xyz, 0.25)


@pytest.mark.parametrize("d", [100.0, 30.0, 1.0 / 2048, 1.0 / 1024, 0.0009765625 * 3.5])
def test_extreme_radii(ctx, d):
    c = synth.blobs_20k()
    assert_parity(ctx, c.xyz, d)


def test_wide_arithmetic_path(ctx):
    """R > 26753 units (d > 26 m) uses 64-bit distance arithmetic."""
    rng = np.random.default_rng(9)
    xyz = synth.to_grid(rng.uniform(-2000, 2000, size=(5000, 3)))
    assert_parity(ctx, xyz, 150.0)
    assert_parity(ctx, xyz, 27.5)


def test_duplicates_and_tiny(ctx):
    xyz = np.zeros((5000, 3), np.float32)
    _, k = assert_parity(ctx, xyz, 0.1)
    assert k == 1
    assert_parity(ctx, xyz[:1], 0.1)
    assert_parity(ctx, xyz[:2], 0.1, 3, 5)


def test_empty(ctx):
    lab, k = run_gpu(ctx, np.zeros((0, 3), np.float32), 0.5, device=False)
    assert k == 0 and lab.size == 0


# ------------------------------------------------------------------ errors

def test_errors(ctx):
    x = np.zeros((100, 3), np.float32)
    for bad, want in [(np.nan, "FEC_ERR_NONFINITE"), (np.inf, "FEC_ERR_NONFINITE"),
                      (8192.0, "FEC_ERR_OUT_OF_RANGE"), (-9000.0, "FEC_ERR_OUT_OF_RANGE")]:
        y = x.copy()
        y[7, 1] = bad
        with pytest.raises(fec.FecError) as e:
            run_gpu(ctx, y, 0.5)
        assert e.value.name == want
    y = x.copy()
    y[3, 0] = 9000.0
    y[50, 2] = np.nan
    with pytest.raises(fec.FecError) as e:
        run_gpu(ctx, y, 0.5)
    assert e.value.name == "FEC_ERR_NONFINITE"
    for d, mn, mx in [(0.0, 1, 2), (-1.0, 1, 2), (float("nan"), 1, 2), (0.5, 3, 2), (0.5, -1, 2)]:
        with pytest.raises(fec.FecError) as e:
            run_gpu(ctx, x, d, mn, mx)
        assert e.value.name == "FEC_ERR_INVALID_ARG"
    # the context stays usable after errors
    assert_parity(ctx, random_cloud(1, 500), 0.3)


def test_budget_oom():
    small = fec.Context(device=0, mem_budget_bytes=1 << 20)
    try:
        with pytest.raises(fec.FecError) as e:
            small.cluster(random_cloud(2, 200_000), 0.3)
        assert e.value.name == "FEC_ERR_OOM"
    finally:
        small.close()


# ------------------------------------------------------------- invariants

def test_determinism_and_permutation(ctx):
    c = synth.frame_120k()
    a, ka = run_gpu(ctx, c.xyz, c.d, c.min_size, c.max_size)
    b, kb = run_gpu(ctx, c.xyz, c.d, c.min_size, c.max_size)
    np.testing.assert_array_equal(a, b)
    perm = np.random.default_rng(3).permutation(c.n)
    p, kp = assert_parity(ctx, c.xyz[perm], c.d, c.min_size, c.max_size)
    assert kp == ka
    check_labels_valid(c.xyz[perm], c.d, p, kp, c.min_size, c.max_size)


def test_translation_by_grid_multiple(ctx):
    c = synth.blobs_20k()
    a, _ = run_gpu(ctx, c.xyz, c.d)
    moved = (c.xyz.astype(np.float64) + np.array([123.0, -7.5, 0.0009765625 * 77])).astype(np.float32)
    b, _ = run_gpu(ctx, moved, c.d)
    np.testing.assert_array_equal(a, b)


def test_stats(ctx):
    c = synth.frame_120k()
    run_gpu(ctx, c.xyz, c.d, c.min_size, c.max_size)
    s = ctx.stats()
    assert s["n"] == c.n and 0 < s["cells"] <= s["subcells"] <= c.n
    assert s["R"] == 358 and s["h"] == 179 and s["T2"] == oracle.threshold(c.d)


@pytest.mark.parametrize("d", [0.05, 0.2, 0.35, 1.0, 3.0])
def test_pairs_across_cell_and_subcell_boundaries(ctx, d):
    """Exercises the geometric shortcuts of the union step (sub-cell cliques,
    the rule that sub-cells three sub-cell steps apart cannot join, box and
    representative tests) exactly at the threshold: every pair must be
    joined iff its squared distance is at most T2."""
    xyz, joined = boundary_pairs(d, seed=int(d * 1000))
    got, k = assert_parity(ctx, xyz, d)
    m = len(joined)
    assert k == int(joined.sum()) + 2 * int((~joined).sum())
    same = got[:m] == got[m:]
    np.testing.assert_array_equal(same, joined)
