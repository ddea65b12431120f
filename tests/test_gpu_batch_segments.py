"""The batch path runs every group of frames that share a radius as one pass
of the pipeline (a sort segmented by frame, a cell table that starts a new
cell at every frame, size bounds and numbering per frame).  These cases aim
at the seams of that design; each frame's labels must equal the oracle on the
frame alone (exact, tolerance 0):

* frames of 1 to 9 points next to each other (several frame starts inside
  one thread's positions of the cell-table scan), and frames of one and two
  sort tiles (2,560 and 5,120 points) and one more or less;
* identical frames (the same coordinates in every frame: cells of different
  frames coincide in space and must never join);
* more frames than one block of the planning kernel handles at once (300),
  and more than one call holds (4,100 frames of one radius: two groups);
* radii interleaved along the input, frames whose first row is not a
  multiple of four (unaligned vector loads), empty frames between them;
* a radius above 1 m (cells wider than 1,024 units: keys are stored and the
  cell table gathers coordinates by input row)."""
import numpy as np
import pytest

import oracle
from paper_2208_07678_gb300 import fec, synth

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


def _check(ctx, frames, d, mn=None, mx=None, device=True):
    import torch

    nb = len(frames)
    mn = [1] * nb if mn is None else mn
    mx = [fec.INT64_MAX] * nb if mx is None else mx
    offs = np.zeros(nb + 1, np.int64)
    offs[1:] = np.cumsum([len(f) for f in frames])
    xyz = np.concatenate([np.asarray(f, np.float32).reshape(-1, 3) for f in frames]) if offs[-1] else \
        np.zeros((0, 3), np.float32)
    x = torch.from_numpy(xyz).cuda() if device else xyz
    labels, ks = ctx.cluster_batch(x, offs, d, mn, mx)
    if device:
        labels = labels.cpu().numpy()
    want = oracle.cluster_many([(f, d[i], mn[i], mx[i]) for i, f in enumerate(frames) if len(f)])
    j = 0
    for i, f in enumerate(frames):
        got = labels[offs[i]:offs[i + 1]]
        if len(f) == 0:
            assert ks[i] == 0
            continue
        w, kw = want[j]
        j += 1
        assert ks[i] == kw, (i, ks[i], kw)
        np.testing.assert_array_equal(got, w, err_msg=f"frame {i}")
    return labels, ks


def _blob(rng, n, scale=1.0):
    return synth.to_grid(rng.normal(0.0, scale, size=(n, 3)))


def test_tiny_frames_side_by_side(ctx):
    rng = np.random.default_rng(101)
    frames = [_blob(rng, 1 + i % 9, 0.2) for i in range(200)]
    _check(ctx, frames, [0.3] * len(frames))
    _check(ctx, frames, [0.3] * len(frames), device=False)


def test_frames_at_sort_tile_sizes(ctx):
    rng = np.random.default_rng(102)
    sizes = [2560, 2561, 2559, 5120, 5121, 5119, 10240, 1, 2560]
    frames = [_blob(rng, n, 3.0) for n in sizes]
    _check(ctx, frames, [0.25] * len(frames))


def test_identical_frames_never_join(ctx):
    c = synth.blobs_20k()
    frames = [c.xyz] * 5
    labels, ks = _check(ctx, frames, [c.d] * 5, [c.min_size] * 5, [c.max_size] * 5)
    assert len(set(ks.tolist())) == 1


def test_three_hundred_frames(ctx):
    frames = synth.batch_256(seed=9, n_frames=300, lo=200, hi=3_000)
    _check(ctx, [f.xyz for f in frames], [f.d for f in frames], [5] * 300, [2_000] * 300)


def test_more_frames_than_one_call_holds(ctx):
    rng = np.random.default_rng(103)
    frames = [_blob(rng, 3 + i % 5, 0.5) for i in range(4100)]
    _check(ctx, frames, [0.35] * len(frames))


def test_interleaved_radii_unaligned_rows_and_empty_frames(ctx):
    rng = np.random.default_rng(104)
    frames, d = [], []
    for i in range(40):
        n = [0, 7, 1234, 5, 30_001, 0, 999][i % 7]
        frames.append(_blob(rng, n, 2.0) if n else np.zeros((0, 3), np.float32))
        d.append([0.25, 0.35, 0.5, 0.35][i % 4])
    mn = [1 + (i % 3) for i in range(40)]
    mx = [fec.INT64_MAX if i % 2 else 500 for i in range(40)]
    _check(ctx, frames, d, mn, mx)
    _check(ctx, frames, d, mn, mx, device=False)


def test_wide_cells_gather_path(ctx):
    rng = np.random.default_rng(105)
    frames = [_blob(rng, n, 20.0) for n in (3000, 17, 4000, 1)]
    _check(ctx, frames, [1.5] * 4)


def test_batch_replays_and_shapes(ctx):
    """The same batch twice (graph replay), then a different shape on the same
    context (a new capture, possibly new tuning)."""
    frames = synth.batch_256(seed=10, n_frames=20, lo=2_000, hi=30_000)
    xs = [f.xyz for f in frames]
    d = [f.d for f in frames]
    for _ in range(2):
        _check(ctx, xs, d, [50] * 20, [50_000] * 20)
    _check(ctx, xs[:7], d[:7], [50] * 7, [50_000] * 7)


def test_tuning_file_round_trip(tmp_path):
    """The tuner writes one "key lanes region big tail" line per batch shape to the
    context's cache file; a new context reading that file runs the same batch
    with the stored configuration and gives the same labels."""
    import torch

    from paper_2208_07678_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    frames = synth.batch_256(seed=11, n_frames=12, lo=2_000, hi=20_000)
    xs = [f.xyz for f in frames]
    d = [f.d for f in frames]
    offs = np.zeros(len(xs) + 1, np.int64)
    offs[1:] = np.cumsum([len(x) for x in xs])
    xyz = np.concatenate(xs)
    path = str(tmp_path / "tune.txt")
    with fec.Context(device=0, autotune_cache=path) as c1:
        lab1, k1 = c1.cluster_batch(xyz, offs, d, [20] * 12, [40_000] * 12)
    lines = [l.split() for l in open(path).read().splitlines() if l.strip()]
    assert lines and all(len(l) == 5 for l in lines)
    for _, lanes, region, big, tail in lines:
        assert 1 <= int(lanes) <= 8 and int(region) in (256, 512, 1024)
        assert int(big) in (32, 64, 128) and int(tail) in (1, 2, 4)
    with fec.Context(device=0, autotune_cache=path) as c2:
        lab2, k2 = c2.cluster_batch(xyz, offs, d, [20] * 12, [40_000] * 12)
    np.testing.assert_array_equal(np.asarray(lab1), np.asarray(lab2))
    np.testing.assert_array_equal(np.asarray(k1), np.asarray(k2))
