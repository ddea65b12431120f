"""The seeded input generators (no GPU): determinism, the 1/1024 m grid,
sizes and parameters of the stand-in workloads, and the serving stream."""
import numpy as np
import pytest

from paper_2208_07678_gb300 import synth


def _on_grid(xyz):
    q = xyz.astype(np.float64) * 1024.0
    return np.array_equal(q, np.rint(q))


def test_blobs_20k_is_seeded_and_on_the_grid():
    a, b = synth.blobs_20k(), synth.blobs_20k()
    assert a.n == 20_000 and a.xyz.dtype == np.float32 and a.xyz.shape == (20_000, 3)
    assert np.array_equal(a.xyz, b.xyz)
    assert not np.array_equal(a.xyz, synth.blobs_20k(seed=2).xyz)
    assert _on_grid(a.xyz)
    assert (a.d, a.min_size, a.max_size) == (0.5, 1, synth.INF_SIZE)
    # blob centres and noise in a 40 m cube; Gaussian tails (sigma <= 1.5 m) reach a little past it
    assert np.all((a.xyz > -10.0) & (a.xyz < 50.0))
    assert np.mean((a.xyz >= 0.0) & (a.xyz <= 40.0)) > 0.98


def test_frame_120k_parameters():
    c = synth.frame_120k()
    assert c.n == 120_537 and _on_grid(c.xyz)
    assert (c.d, c.min_size, c.max_size) == (0.35, 50, 50_000)
    r = np.hypot(c.xyz[:, 0], c.xyz[:, 1])
    assert r.max() <= 80.5                      # ground clipped at 80 m (plus range noise)


def test_short_map_is_a_prefix_of_frames():
    m = synth.map_27m(n_frames=2)
    assert _on_grid(m.xyz) and (m.d, m.min_size, m.max_size) == (0.2, 100, 2_000_000)
    crop = synth.map_crop(m, 0.0, 5.0)
    assert np.all((crop.xyz[:, 0] >= 0.0) & (crop.xyz[:, 0] < 5.0))
    assert crop.n == int(np.count_nonzero((m.xyz[:, 0] >= 0.0) & (m.xyz[:, 0] < 5.0)))


def test_serve_stream():
    for i in range(6):
        r = synth.serve_request(5, i)
        assert 10_000 <= r.n <= 2_000_000 and _on_grid(r.xyz)
        assert 0.15 <= r.d <= 0.6 and 10 <= r.min_size <= 200 and r.max_size == synth.INF_SIZE
    t = synth.poisson_arrivals(5, 400.0, 2.0)
    assert np.all(np.diff(t) > 0) and t[-1] < 2.0
    assert 0.8 * 800 < t.size < 1.2 * 800       # about rate x duration arrivals
    assert np.array_equal(t, synth.poisson_arrivals(5, 400.0, 2.0))


def test_batch_frames():
    frames = synth.batch_256(n_frames=5)
    assert len(frames) == 5
    for f in frames:
        assert 20_000 * 0.9 <= f.n <= 180_000 and f.d in (0.25, 0.35, 0.5) and _on_grid(f.xyz)


@pytest.mark.parametrize("n_clusters,density", [(10, 8), (25, 27)])
def test_voxel_clusters_fill_separate_voxels(n_clusters, density):
    xyz = synth.voxel_clusters(3, n_clusters, density)
    assert xyz.shape == (n_clusters * density, 3) and _on_grid(xyz)
    vox = np.floor(xyz.astype(np.float64)).astype(np.int64)
    keys, counts = np.unique(vox, axis=0, return_counts=True)
    assert len(keys) == n_clusters and np.all(counts == density)
    assert np.all(keys % 2 == 0)                # every other lattice site: voxels never touch
