"""fec_cluster_noalloc, the entry point for callers that cannot allocate
device memory (a host application that owns all device memory through its
own pool, a real-time loop, a plug-in that must not call cudaMalloc): its
workspace is a fixed array in the library's device image.  Checked through
the C ABI against fec_cluster on the same clouds, on consecutive calls (the
array keeps the previous call's contents, so the second call must not depend
on them).  Labels are integers with one correct answer: equality is exact.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

from paper_2208_07678_gb300 import fec, synth

pytestmark = pytest.mark.gpu


def _clouds():
    a = synth.blobs_20k()  # 20,000 points, d = 0.5
    rng = np.random.default_rng(77)
    xyz = synth.to_grid(synth.frame_of_size(rng, 30_000))
    b = synth.Cloud(xyz[rng.permutation(len(xyz))], 0.35, 50, 50_000, "frame_30k")
    return [a, b]


def _reference(clouds):
    out = []
    with fec.Context(device=0) as ctx:
        for c in clouds:
            out.append(ctx.cluster(c.xyz, c.d, c.min_size, c.max_size))
    return out


def _noalloc(c, device):
    import torch

    if device:
        x = torch.from_numpy(c.xyz).cuda()
        lab = torch.full((c.n,), -7, dtype=torch.int32, device="cuda")
        st, k = fec.fec_cluster_noalloc(x.data_ptr(), c.n, c.d, c.min_size, c.max_size,
                                        lab.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return st, k, lab.cpu().numpy()
    x = np.ascontiguousarray(c.xyz)
    lab = np.full(c.n, -7, dtype=np.int32)
    st, k = fec.fec_cluster_noalloc(x.ctypes.data, c.n, c.d, c.min_size, c.max_size,
                                    lab.ctypes.data)
    return st, k, lab


@pytest.mark.parametrize("device", [True, False], ids=["device", "host"])
def test_noalloc_equals_fec_cluster_on_consecutive_calls(device):
    import torch

    from paper_2208_07678_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    clouds = _clouds()
    assert all(c.n <= fec.FEC_NOALLOC_MAX_POINTS for c in clouds)
    want = _reference(clouds)
    # two calls in a row on different clouds, then the first cloud again
    for c, (lab_ref, k_ref) in list(zip(clouds, want)) + [(clouds[0], want[0])]:
        st, k, lab = _noalloc(c, device)
        assert fec.STATUS[st] == "FEC_OK"
        assert k == k_ref
        np.testing.assert_array_equal(lab, lab_ref)


def test_noalloc_rejects_clouds_above_its_capacity():
    n = fec.FEC_NOALLOC_MAX_POINTS + 1
    x = np.zeros((n, 3), np.float32)
    lab = np.zeros(n, np.int32)
    st, _ = fec.fec_cluster_noalloc(x.ctypes.data, n, 0.5, 1, 10, lab.ctypes.data)
    assert fec.STATUS[st] == "FEC_ERR_INVALID_ARG"


def test_noalloc_reports_a_cloud_wider_than_its_slab_index():
    """The static workspace's slab index has 65,536 entries, each a row of 16
    grid cells along the major axis (1,048,576 cells): a cloud wider than that
    is refused with FEC_ERR_OUT_OF_RANGE (the device plan sees the overflow
    before any key is sorted), and the next call on an ordinary cloud is
    exact again."""
    import torch

    from paper_2208_07678_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)
    d = 0.005  # cells of 6 units: 1,048,576 of them span 6,144 m
    x = np.array([[-4000.0, 0.0, 0.0], [4000.0, 0.0, 0.0], [4000.0, 0.00390625, 0.0]], np.float32)
    lab = np.full(3, -7, np.int32)
    st, _ = fec.fec_cluster_noalloc(x.ctypes.data, 3, d, 1, fec.INT64_MAX, lab.ctypes.data)
    assert fec.STATUS[st] == "FEC_ERR_OUT_OF_RANGE"
    with fec.Context(device=0) as ctx:
        want, kw = ctx.cluster(x, d, 1, fec.INT64_MAX)
    assert kw == 2  # fec_cluster has no such limit
    c = synth.blobs_20k()
    ref = _reference([c])[0]
    st, k, lab = _noalloc(c, False)
    assert fec.STATUS[st] == "FEC_OK" and k == ref[1]
    np.testing.assert_array_equal(lab, ref[0])


def test_noalloc_reports_boundary_lists_it_cannot_hold():
    """A lattice with one point in every sub-cell (32^3 points, spacing h =
    0.25 m at d = 0.5 m) makes far more joined sub-cell pairs across the
    neighbour step's regions than the fixed lists hold (two entries per
    point).  fec_cluster grows its lists and retries; the static workspace
    cannot, so the call reports FEC_ERR_OOM.  The next ordinary call is exact."""
    import torch

    torch.cuda.set_device(0)
    g = (np.arange(32, dtype=np.float32) + 0.5) * 0.25
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    x = np.ascontiguousarray(x[np.random.default_rng(5).permutation(len(x))])
    n = len(x)
    assert n <= fec.FEC_NOALLOC_MAX_POINTS
    with fec.Context(device=0) as ctx:
        want, kw = ctx.cluster(x, 0.5, 1, fec.INT64_MAX)
    assert kw == 1 and np.all(want == 0)
    lab = np.full(n, -7, np.int32)
    st, _ = fec.fec_cluster_noalloc(x.ctypes.data, n, 0.5, 1, fec.INT64_MAX, lab.ctypes.data)
    assert fec.STATUS[st] == "FEC_ERR_OOM"
    c = synth.blobs_20k()
    ref = _reference([c])[0]
    st, k, lab = _noalloc(c, True)
    assert fec.STATUS[st] == "FEC_OK" and k == ref[1]
    np.testing.assert_array_equal(lab, ref[0])


def test_noalloc_after_device_reset(tmp_path):
    """The cached workspace address belongs to the context it was taken in.
    A separate process (sharing the library's CUDA runtime: it links the
    library's objects) calls the entry point, resets the device, and calls it
    again: the second call must redo its set-up in the new context and give
    the same labels.  Run once, on a 4,000-point cloud."""
    import glob
    import os
    import subprocess

    from paper_2208_07678_gb300 import build as libbuild

    libbuild.build()
    here = os.path.dirname(os.path.abspath(__file__))
    objs = sorted(glob.glob(os.path.join(libbuild.BUILD, "*.o")))
    exe = str(tmp_path / "noalloc_reset")
    cmd = [libbuild.nvcc(), *libbuild.ARCH, "-O2", "-std=c++17", "-I", libbuild.INCLUDE,
           os.path.join(here, "noalloc_reset.cu"), *objs, "-lpthread", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "labels equal" in r.stdout
