"""Failure detection on the device, without a fault: the device loops that
wait on other blocks (look-back of the sort and of the cell-table scan) and
the loops that walk the global union-find are bounded.  A test lowers those
bounds through fec_set_iteration_caps so that a wait or a union runs out on
purpose (no flag that anything would set is needed: with a cap of 0 the first
wait or walk gives up), and checks what the caller sees:

* FEC_ERR_NOT_CONVERGED, or FEC_OK with labels equal to the oracle's -- never
  FEC_OK with wrong labels;
* the context stays usable: with the default caps back, the next call on the
  same context is exact again.

Labels are integers with one correct answer, so comparisons are exact."""
import numpy as np
import pytest

import oracle
from paper_2208_07678_gb300 import fec, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frame():
    c = synth.frame_120k()
    want = oracle.cluster(c.xyz, c.d, c.min_size, c.max_size)
    return c, want


@pytest.fixture(scope="module")
def corridor():
    # ten corridor frames (about 1.2M points): hundreds of sort tiles, so the
    # look-back of some tile finds its predecessor not yet published
    c = synth.map_27m(n_frames=10)
    want = oracle.cluster(c.xyz, c.d, c.min_size, c.max_size)
    return c, want


def _run(ctx, c, device):
    import torch

    x = torch.from_numpy(c.xyz).cuda() if device else c.xyz
    try:
        lab, k = ctx.cluster(x, c.d, c.min_size, c.max_size)
    except fec.FecError as e:
        return e.name, None, None
    if device:
        lab = lab.cpu().numpy()
    return "FEC_OK", lab, k


def _lib():
    import torch

    from paper_2208_07678_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(0)


def test_union_cap_run_out_is_reported_and_context_recovers(frame):
    """The frame's ground spans many regions of the neighbour step, so the
    boundary unions are certain to run: with a union cap of 0 every one of
    them gives up, and the call must say so."""
    _lib()
    c, (want, kw) = frame
    with fec.Context(device=0) as ctx:
        ctx.set_iteration_caps(fec.FEC_DEFAULT_WAIT_CAP, 0)
        for device in (True, False):
            st, _, _ = _run(ctx, c, device)
            assert st == "FEC_ERR_NOT_CONVERGED"
        ctx.set_iteration_caps()
        st, lab, k = _run(ctx, c, True)
        assert st == "FEC_OK" and k == kw
        np.testing.assert_array_equal(lab, want)


def test_wait_cap_run_out_never_returns_wrong_labels(corridor):
    """A wait cap of 0 makes the first look-back that finds its predecessor
    unpublished give up; every later kernel of the call then returns at once.
    Each run is either reported or exact, and over a few runs at least one
    wait gives up."""
    _lib()
    c, (want, kw) = corridor
    seen = []
    with fec.Context(device=0) as ctx:
        ctx.set_iteration_caps(0, fec.FEC_DEFAULT_UNION_CAP)
        for _ in range(3):
            st, lab, k = _run(ctx, c, True)
            seen.append(st)
            assert st in ("FEC_OK", "FEC_ERR_NOT_CONVERGED")
            if st == "FEC_OK":
                assert k == kw
                np.testing.assert_array_equal(lab, want)
        assert "FEC_ERR_NOT_CONVERGED" in seen
        ctx.set_iteration_caps()
        st, lab, k = _run(ctx, c, True)
        assert st == "FEC_OK" and k == kw
        np.testing.assert_array_equal(lab, want)


def test_both_caps_zero_then_defaults(frame):
    _lib()
    c, (want, kw) = frame
    with fec.Context(device=0) as ctx:
        ctx.set_iteration_caps(0, 0)
        st, _, _ = _run(ctx, c, True)
        assert st == "FEC_ERR_NOT_CONVERGED"
        ctx.set_iteration_caps()
        for device in (True, False):
            st, lab, k = _run(ctx, c, device)
            assert st == "FEC_OK" and k == kw
            np.testing.assert_array_equal(lab, want)
