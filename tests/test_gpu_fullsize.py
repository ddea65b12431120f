"""Full-size parity on the accumulated 27.9M-point corridor map, in the same
call bench.py times (device-resident input through fec_cluster).  The oracle
runs in a background thread (ctypes releases the GIL) while the GPU works."""
import threading

import numpy as np
import pytest

import oracle
from paper_2208_07678_gb300 import fec, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_map_27m_bit_exact():
    import torch

    from paper_2208_07678_gb300 import build as libbuild

    libbuild.build()
    cloud = synth.map_27m()
    want = {}

    def run_oracle():
        want["labels"], want["k"] = oracle.cluster(cloud.xyz, cloud.d, cloud.min_size, cloud.max_size)

    th = threading.Thread(target=run_oracle)
    th.start()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    with fec.Context(device=0, cuda_stream=stream.cuda_stream) as ctx:
        xyz = torch.from_numpy(cloud.xyz).cuda()
        lab = torch.empty(cloud.n, dtype=torch.int32, device="cuda")
        _, k = ctx.cluster(xyz, cloud.d, cloud.min_size, cloud.max_size, labels=lab)
        _, k2 = ctx.cluster(xyz, cloud.d, cloud.min_size, cloud.max_size, labels=lab)
        got = lab.cpu().numpy()
        stats = ctx.stats()
    th.join()
    assert k == k2 == want["k"]
    bad = np.nonzero(got != want["labels"])[0]
    assert bad.size == 0, f"{bad.size} of {cloud.n} labels differ, first {bad[:8]}"
    assert stats["n"] == cloud.n and stats["key_bits"] <= 32
    # dense numbering 0..k-1 by smallest index, sizes within the bounds
    kept = got[got >= 0]
    sizes = np.bincount(kept, minlength=k)
    assert sizes.min() >= cloud.min_size and sizes.max() <= cloud.max_size
    first = np.full(k, cloud.n, np.int64)
    np.minimum.at(first, kept, np.nonzero(got >= 0)[0])
    assert np.all(np.diff(first) > 0)
