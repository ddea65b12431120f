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
