"""Oracle parity at the stated sizes of the batched and the serving workloads.

* Batch: the full 256-frame workload (frames of 20k-180k points, log-uniform;
  d per frame from {0.25, 0.35, 0.5} m; min 50, max 50,000) in one
  fec_cluster_batch call with device-resident input, the call the bench
  times; every frame's labels are compared element by element with the oracle
  on that frame alone (frame-local numbering).
* Serving: a mix of twelve requests from the serving stream (10k-2M points,
  one of them above 1.8M), with d at both ends of [0.15, 0.6] m and
  min_size at both ends of [10, 200] among them, all submitted before the
  first poll so that they overlap on the device; each result is compared
  with the oracle and with fec_cluster on that request alone.

The oracle runs in a pool of worker processes (spawn), one cloud per task.
Labels are integers with one correct answer: equality is exact."""
import numpy as np
import pytest

import oracle
from paper_2208_07678_gb300 import fec, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _lib():
    import torch

    from paper_2208_07678_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def batch():
    frames = synth.batch_256()
    want = oracle.cluster_many([(f.xyz, f.d, f.min_size, f.max_size) for f in frames])
    return frames, want


def test_batch_256_equals_oracle(batch):
    import torch

    _lib()
    frames, want = batch
    assert len(frames) == 256
    sizes = np.array([f.n for f in frames])
    assert sizes.min() >= 20_000 and sizes.max() <= 180_000
    assert set(f.d for f in frames) == {0.25, 0.35, 0.5}
    offs = np.zeros(len(frames) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    xyz = torch.from_numpy(np.concatenate([f.xyz for f in frames])).cuda()
    lab = torch.full((int(offs[-1]),), -7, dtype=torch.int32, device="cuda")
    d = [f.d for f in frames]
    mn = [f.min_size for f in frames]
    mx = [f.max_size for f in frames]
    with fec.Context(device=0, cuda_stream=torch.cuda.current_stream().cuda_stream) as ctx:
        for rep in range(2):  # the second call replays the captured batch
            lab.fill_(-7)
            _, ks = ctx.cluster_batch(xyz, offs, d, mn, mx, labels=lab)
            got = lab.cpu().numpy()
            for f in range(len(frames)):
                w, kw = want[f]
                assert ks[f] == kw, (rep, f)
                g = got[offs[f]:offs[f + 1]]
                bad = np.nonzero(g != w)[0]
                assert bad.size == 0, f"call {rep}, frame {f}: {bad.size} labels differ"


def _serve_mix():
    reqs = [synth.serve_request(5, i) for i in range(12)]
    # the ends of the stated ranges: d in [0.15, 0.6], min_size in [10, 200]
    big = max(range(12), key=lambda i: reqs[i].n)
    small = min(range(12), key=lambda i: reqs[i].n)
    reqs[big].d = float(np.float32(0.15))
    reqs[small].d = float(np.float32(0.6))
    reqs[big].min_size = 10
    reqs[small].min_size = 200
    mid = [i for i in range(12) if i not in (big, small)][0]
    reqs[mid].d = float(np.float32(0.6))
    return reqs


def test_serve_mix_equals_oracle_alone_and_in_mix():
    reqs = _serve_mix()
    assert max(r.n for r in reqs) >= 1_500_000 and min(r.n for r in reqs) <= 50_000
    assert min(r.d for r in reqs) == pytest.approx(0.15) and max(r.d for r in reqs) == pytest.approx(0.6)
    want = oracle.cluster_many([(r.xyz, r.d, r.min_size, r.max_size) for r in reqs])
    _lib()
    with fec.Context(device=0) as srv, fec.Context(device=0) as solo:
        outs = [np.full(r.n, -7, np.int32) for r in reqs]
        tickets = [srv.submit(r.xyz, r.d, r.min_size, r.max_size, o) for r, o in zip(reqs, outs)]
        for i, (r, o, t) in enumerate(zip(reqs, outs, tickets)):
            st, k = srv.poll(t, -1)
            assert st == fec.FEC_OK, (i, fec.STATUS[st])
            w, kw = want[i]
            assert k == kw, i
            np.testing.assert_array_equal(o, w)
            alone, k_alone = solo.cluster(r.xyz, r.d, r.min_size, r.max_size)
            assert k_alone == kw
            np.testing.assert_array_equal(alone, w)
