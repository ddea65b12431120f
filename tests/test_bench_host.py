"""Host-side logic of bench.py (no GPU): clock-sample summaries, the guard on
committed DRAM-traffic figures, the algorithmic-byte table, the bounded
oracle sample and the submit/poll loop of the pipelined end-to-end figure."""
import importlib.util
import json
import os
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _sample_line(ts, sm, sm_max, power_cap="Not Active", hw="Not Active"):
    stamp = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(ts)) + ".%03d" % int((ts % 1) * 1000)
    return f"{stamp}, 0, {sm}, {sm_max}, 900.5, 0x0, {hw}, Not Active, Not Active, {power_cap}\n"


def test_clock_summary_keeps_samples_inside_timed_windows(bench, tmp_path):
    now = time.time()
    p = tmp_path / "clocks.csv"
    p.write_text(_sample_line(now - 10, 1200, 2070) +              # warm-up, outside
                 _sample_line(now + 0.1, 2070, 2070) +
                 _sample_line(now + 0.2, 2055, 2070, power_cap="Active") +
                 _sample_line(now + 0.3, 2070, 2070) +
                 _sample_line(now + 20, 900, 2070, hw="Active"))   # after, outside
    cs = bench.ClockSampler(0)
    cs.path = str(p)
    cs.mark(now, now + 1.0)
    s = cs.summary()
    assert s["samples"] == 3 and s["window"] == "timed steps"
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]   # hw_slowdown was outside the window
    assert not p.exists()                      # the temporary file is removed


def test_clock_summary_without_samples_in_window_says_so(bench, tmp_path):
    now = time.time()
    p = tmp_path / "clocks.csv"
    p.write_text(_sample_line(now - 5, 1800, 2070) + _sample_line(now - 4, 1900, 2070))
    cs = bench.ClockSampler(0)
    cs.path = str(p)
    cs.mark(now, now + 1.0)
    s = cs.summary()
    assert s["samples"] == 2 and s["window"].startswith("whole measurement")
    assert s["sm_mhz"] == 1850.0


def test_clock_summary_unsampled(bench):
    cs = bench.ClockSampler(0)
    assert cs.summary()["reasons"] == ["unsampled"]


def test_traffic_is_dropped_once_the_kernel_source_changes(bench, monkeypatch):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        j = json.load(f)
    entry = j["map_27m"]["k_region"]
    monkeypatch.setattr(bench, "source_hash", lambda fname: entry["source_sha"])
    assert bench.ncu_traffic("k_region", "map_27m") == entry["bytes_per_launch"]
    monkeypatch.setattr(bench, "source_hash", lambda fname: "0" * 16)
    assert bench.ncu_traffic("k_region", "map_27m") is None
    assert bench.ncu_traffic("k_region", "no_such_workload") is None


def test_committed_traffic_is_consistent_with_the_algorithmic_bytes(bench):
    """The full-map figure is the small capture scaled by the algorithmic
    bytes; both sit a little above those bytes (no gross re-reads)."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        j = json.load(f)
    # sizes of the two workloads (cells, sub-cells), as the bench reports them
    small = bench.KERNEL_BYTES["k_region"](12_141_972, 2_373_102, 833_547)
    full = bench.KERNEL_BYTES["k_region"](27_930_995, 5_459_358, 1_895_339)
    ts, tf = j["map_frames:100"]["k_region"]["bytes_per_launch"], j["map_27m"]["k_region"]["bytes_per_launch"]
    assert 1.0 <= ts / small <= 1.5
    assert tf == pytest.approx(ts * full / small, rel=1e-6)


def test_algorithmic_bytes_table(bench):
    kb = bench.KERNEL_BYTES
    n, Ms, Mc = 1000, 300, 100
    assert kb["k_region"](n, Ms, Mc) == 88 * Mc + 40 * Ms   # cell 88; box 32, rep 4, parent 4
    assert kb["onesweep_u32"](n, Ms, Mc) == 24 * n       # key 4 + payload 8, read and written
    assert kb["k_keys"](n, Ms, Mc) == 12 * n             # coordinates read, histograms only
    for name, f in kb.items():
        assert f(2 * n, 2 * Ms, 2 * Mc) == 2 * f(n, Ms, Mc), name   # linear in the sizes
        assert name in bench.KERNEL_SOURCE


def test_oracle_sample_is_a_bounded_density_preserving_crop(bench):
    from paper_2208_07678_gb300 import synth

    cloud = synth.map_27m(n_frames=24)   # long enough for the density to be even along x
    sample, desc = bench.oracle_sample(cloud, cloud.n // 4)
    assert 0 < sample.n < cloud.n and "x-window crop" in desc
    assert 0.5 * cloud.n / 4 < sample.n < 2.0 * cloud.n / 4
    x = sample.xyz[:, 0]
    assert np.all((x >= x.min()) & (x <= x.max()))
    whole, desc2 = bench.oracle_sample(cloud, cloud.n + 1)
    assert whole is cloud and desc2.startswith("whole cloud")


def test_unknown_workload_is_refused(bench):
    with pytest.raises(SystemExit):
        bench.make_workload("no_such_workload")


def test_host_info_and_all_core_batch_baseline():
    import bench
    from paper_2208_07678_gb300 import synth

    info = bench.host_info()
    assert info["nproc"] >= 1 and isinstance(info["cpu_model"], str) and info["cpu_model"]
    frames = synth.batch_256(seed=8, n_frames=3, lo=500, hi=1_000)
    out = bench.time_oracle_batch(frames, processes=2)
    assert out["frames_per_s"] > 0 and out["cores"] == 2 and out["kind"] == "oracle"


class _FakeBuffer:
    _next = 0x1000

    def __init__(self):
        _FakeBuffer._next += 0x100
        self.ptr = _FakeBuffer._next

    def pin_memory(self):
        return self

    def data_ptr(self):
        return self.ptr


class _FakeTorch:
    int32 = "int32"

    @staticmethod
    def empty(n, dtype=None):
        return _FakeBuffer()

    class cuda:
        @staticmethod
        def synchronize(dev=None):
            pass


class _FakeFec:
    """Records the submit/poll sequence of the pipelined end-to-end loop."""
    FEC_OK = 0
    STATUS = {0: "FEC_OK"}

    class FecError(RuntimeError):
        def __init__(self, st, where=""):
            super().__init__(where)

    def __init__(self):
        self.in_flight = {}   # ticket -> label buffer
        self.max_in_flight = 0
        self.events = []
        self.next_ticket = 1
        fake = self

        class Context:
            def __init__(self, device=0):
                self.handle = 7

            def __enter__(self):
                return self

            def __exit__(self, *a):
                return False

            def poll(self, t, timeout_ms=-1):
                fake.events.append(("poll", t))
                del fake.in_flight[t]
                return 0, 42

        self.Context = Context

    def fec_serve_submit(self, handle, xyz, n, d, mn, mx, out):
        assert out not in self.in_flight.values(), "a label buffer reused while its request is in flight"
        t = self.next_ticket
        self.next_ticket += 1
        self.in_flight[t] = out
        self.max_in_flight = max(self.max_in_flight, len(self.in_flight))
        self.events.append(("submit", t))
        return 0, t


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipelined_e2e_keeps_depth_in_flight_and_never_reuses_a_busy_buffer(bench, depth):
    from types import SimpleNamespace

    fake = _FakeFec()
    cloud = SimpleNamespace(n=1000, d=0.2, min_size=1, max_size=10)
    r = bench.measure_e2e_pipelined(fake, _FakeTorch, SimpleNamespace(index=0), cloud, _FakeBuffer(),
                                    steps=7, warmup=3, depth=depth)
    assert fake.max_in_flight == depth and not fake.in_flight
    submits = [t for e, t in fake.events if e == "submit"]
    polls = [t for e, t in fake.events if e == "poll"]
    assert polls == submits  # every request completed, oldest first
    assert r["h2d_bytes_per_step"] == 12 * 1000 and r["d2h_bytes_per_step"] == 4 * 1000 + 4
    assert r["k"] == 42 and r["value"] > 0 and f"{depth} clouds in flight" in r["api"]
