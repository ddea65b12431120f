"""Batched and served clustering: every frame's / request's labels equal the
one-cloud call on that cloud alone (exact, tolerance 0), and match the
oracle."""
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


def small_batch(n_frames=12, seed=41):
    frames = synth.batch_256(seed=seed, n_frames=n_frames, lo=2_000, hi=40_000)
    offs = np.zeros(n_frames + 1, np.int64)
    offs[1:] = np.cumsum([f.n for f in frames])
    xyz = np.concatenate([f.xyz for f in frames])
    return frames, offs, xyz


@pytest.mark.parametrize("device", [True, False], ids=["device", "host"])
def test_batch_equals_single_and_oracle(ctx, device):
    import torch

    frames, offs, xyz = small_batch()
    d = [f.d for f in frames]
    mn = [f.min_size for f in frames]
    mx = [f.max_size for f in frames]
    x = torch.from_numpy(xyz).cuda() if device else xyz
    labels, ks = ctx.cluster_batch(x, offs, d, mn, mx)
    if device:
        labels = labels.cpu().numpy()
    for f, fr in enumerate(frames):
        got = labels[offs[f]:offs[f + 1]]
        alone, k_alone = ctx.cluster(fr.xyz, fr.d, fr.min_size, fr.max_size)
        want, kw = oracle.cluster(fr.xyz, fr.d, fr.min_size, fr.max_size)
        assert ks[f] == k_alone == kw
        np.testing.assert_array_equal(got, alone)
        np.testing.assert_array_equal(got, want)


def test_batch_with_empty_frames(ctx):
    frames, offs, xyz = small_batch(4, seed=43)
    # insert empty frames at the start, middle and end
    offs2 = np.array([0, 0, offs[1], offs[2], offs[2], offs[3], offs[4], offs[4]], np.int64)
    src = [None, 0, 1, None, 2, 3, None]
    d = [0.3 if s is None else frames[s].d for s in src]
    labels, ks = ctx.cluster_batch(xyz, offs2, d, [50] * 7, [50_000] * 7)
    for f, s in enumerate(src):
        if s is None:
            assert ks[f] == 0
            continue
        want, kw = oracle.cluster(frames[s].xyz, frames[s].d, 50, 50_000)
        assert ks[f] == kw
        np.testing.assert_array_equal(labels[offs2[f]:offs2[f + 1]], want)


def test_batch_error_in_one_frame(ctx):
    frames, offs, xyz = small_batch(3, seed=44)
    bad = xyz.copy()
    bad[offs[1] + 5, 0] = np.nan
    with pytest.raises(fec.FecError) as e:
        ctx.cluster_batch(bad, offs, [f.d for f in frames], [1] * 3, [fec.INT64_MAX] * 3)
    assert e.value.name == "FEC_ERR_NONFINITE"


def test_serve_results_equal_alone():
    """Requests submitted together overlap on the device; each result is the
    same as clustering that request alone."""
    reqs = [synth.serve_request(5, i, lo=5_000, hi=400_000) for i in range(10)]
    with fec.Context(device=0) as srv, fec.Context(device=0) as solo:
        outs = [np.full(r.n, -7, np.int32) for r in reqs]
        tickets = [srv.submit(r.xyz, r.d, r.min_size, r.max_size, o) for r, o in zip(reqs, outs)]
        for r, o, t in zip(reqs, outs, tickets):
            st, k = srv.poll(t, -1)
            assert st == fec.FEC_OK
            alone, k_alone = solo.cluster(r.xyz, r.d, r.min_size, r.max_size)
            assert k == k_alone
            np.testing.assert_array_equal(o, alone)
        # oracle on two of them
        for r, o in list(zip(reqs, outs))[:2]:
            want, _ = oracle.cluster(r.xyz, r.d, r.min_size, r.max_size)
            np.testing.assert_array_equal(o, want)


def test_serve_poll_semantics():
    with fec.Context(device=0) as srv:
        r = synth.serve_request(5, 3, lo=50_000, hi=60_000)
        out = np.zeros(r.n, np.int32)
        t = srv.submit(r.xyz, r.d, r.min_size, r.max_size, out)
        st, _ = srv.poll(t, -1)
        assert st == fec.FEC_OK
        st, _ = srv.poll(t, 0)  # released
        assert fec.STATUS[st] == "FEC_ERR_INVALID_ARG"


def test_serve_completion_time():
    """poll_timed reports when the request's result was final, on the clock
    of time.perf_counter (CLOCK_MONOTONIC): after the submit started and
    before the poll returned; the input buffer may change right after submit."""
    import time

    with fec.Context(device=0) as srv, fec.Context(device=0) as solo:
        r = synth.serve_request(5, 4, lo=100_000, hi=120_000)
        xyz = r.xyz.copy()
        out = np.zeros(r.n, np.int32)
        t_submit = time.perf_counter()
        t = srv.submit(xyz, r.d, r.min_size, r.max_size, out)
        xyz[:] = 0.0  # the engine copied the input before submit returned
        st, k, done_ns = srv.poll_timed(t, -1)
        t_after = time.perf_counter()
        assert st == fec.FEC_OK
        assert t_submit <= done_ns * 1e-9 <= t_after
        want, k_want = solo.cluster(r.xyz, r.d, r.min_size, r.max_size)
        assert k == k_want
        np.testing.assert_array_equal(out, want)


def test_serve_rejects_over_budget():
    with fec.Context(device=0, mem_budget_bytes=1 << 20) as srv:
        xyz = np.zeros((100_000, 3), np.float32)
        with pytest.raises(fec.FecError) as e:
            srv.submit(xyz, 0.3, 1, 10, np.zeros(100_000, np.int32))
        assert e.value.name == "FEC_ERR_BUSY"


def test_serve_deadline_drops_requests_that_cannot_start():
    """A request whose deadline passes before a slot takes it completes with
    FEC_ERR_TIMEOUT without running (labels untouched); the requests around
    it are unaffected."""
    big = [synth.serve_request(5, i, lo=300_000, hi=400_000) for i in range(6)]
    small = synth.serve_request(5, 20, lo=5_000, hi=6_000)
    with fec.Context(device=0) as srv, fec.Context(device=0) as solo:
        outs = [np.full(r.n, -7, np.int32) for r in big]
        tickets = [srv.submit(r.xyz, r.d, r.min_size, r.max_size, o) for r, o in zip(big, outs)]
        late = np.full(small.n, -7, np.int32)
        t_late = srv.submit(small.xyz, small.d, small.min_size, small.max_size, late, deadline_us=1)
        st, _ = srv.poll(t_late, -1)
        assert fec.STATUS[st] == "FEC_ERR_TIMEOUT"
        assert np.all(late == -7)
        for r, o, t in zip(big, outs, tickets):
            st, k = srv.poll(t, -1)
            assert st == fec.FEC_OK
            alone, k_alone = solo.cluster(r.xyz, r.d, r.min_size, r.max_size)
            assert k == k_alone
            np.testing.assert_array_equal(o, alone)
        # a generous deadline does not drop anything
        ok = np.full(small.n, -7, np.int32)
        t_ok = srv.submit(small.xyz, small.d, small.min_size, small.max_size, ok, deadline_us=10_000_000)
        st, k = srv.poll(t_ok, -1)
        assert st == fec.FEC_OK
        want, kw = oracle.cluster(small.xyz, small.d, small.min_size, small.max_size)
        assert k == kw
        np.testing.assert_array_equal(ok, want)
        s = srv.serve_stats()
        assert s["expired"] == 1 and s["completed"] == 7 and s["submitted"] == 8


def test_serve_queue_full_is_busy_and_accepted_requests_are_exact():
    """With a 64 MiB budget the input arena holds about eleven 120k-point
    inputs and only one request runs at a time; forty submits in a row from
    device memory fill the arena, and the surplus is refused with
    FEC_ERR_BUSY (no ticket).  Every accepted request is exact."""
    import torch

    c = synth.frame_120k()
    want, kw = oracle.cluster(c.xyz, c.d, c.min_size, c.max_size)
    x = torch.from_numpy(c.xyz).cuda()
    torch.cuda.synchronize()
    with fec.Context(device=0, mem_budget_bytes=64 << 20) as srv:
        outs, tickets, busy = [], [], 0
        for _ in range(40):
            o = np.full(c.n, -7, np.int32)
            st, t = fec.fec_serve_submit(srv.handle, x.data_ptr(), c.n, c.d, c.min_size, c.max_size,
                                         o.ctypes.data)
            if fec.STATUS[st] == "FEC_ERR_BUSY":
                busy += 1
                continue
            assert st == fec.FEC_OK
            outs.append(o)
            tickets.append(t)
        for o, t in zip(outs, tickets):
            st, k = srv.poll(t, -1)
            assert st == fec.FEC_OK and k == kw
            np.testing.assert_array_equal(o, want)
        s = srv.serve_stats()
        assert busy >= 1 and s["rejected"] == busy
        assert s["arena_bytes"] == 16 << 20 and s["queue_max"] >= 2
