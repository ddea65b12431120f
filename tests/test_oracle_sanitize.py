"""The oracle under the host address and undefined-behaviour sanitizers.

``oracle/fec_oracle.c`` and the driver ``tests/oracle_sanitize_main.c`` are
compiled with ``-fsanitize=address,undefined -fno-sanitize-recover=all`` into
one executable, which reads cases produced by the seeded generators
(``paper_2208_07678_gb300.synth``; plain numpy, so the sanitizers have nothing
to instrument there) and runs both oracle routes on each: the kd-tree BFS on
every case, the all-pairs union-find on the small ones.  The test passes when
the process exits cleanly (no sanitizer report), the BFS results equal those
of the oracle built normally, and the two routes agree.

Cases: empty and one-point clouds, 64 copies of one point, the generators'
blobs, Section 3.3.1 voxel clusters and a crop of a LiDAR frame, a long chain
of points exactly d apart, the largest coordinate in range, and the argument
and data errors (d <= 0, min > max, NaN, a coordinate out of range)."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle
from paper_2208_07678_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
FLAGS = ["-O1", "-g", "-std=c11", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
         "-fno-sanitize-recover=all"]


def _fnv(labels):
    h = 1469598103934665603
    for b in np.ascontiguousarray(labels, np.int32).tobytes():
        h ^= b
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _cases():
    rng = np.random.default_rng(77)
    big = 2**63 - 1
    c = []
    c.append(("empty", np.zeros((0, 3), np.float32), 0.5, 1, big, 1))
    c.append(("one point", np.array([[1.0, 2.0, 3.0]], np.float32), 0.5, 1, big, 1))
    c.append(("64 copies", np.tile(np.array([[0.25, -7.5, 3.0]], np.float32), (64, 1)), 0.2, 1, big, 1))
    c.append(("blob 1500", synth.to_grid(rng.normal(0, 1.0, (1500, 3))), 0.25, 3, 400, 1))
    c.append(("voxel 40x20", synth.voxel_clusters(5, 40, 20), 0.1, 1, big, 1))
    f = synth.frame_120k()
    c.append(("frame crop 20k", f.xyz[:20_000], f.d, f.min_size, f.max_size, 0))
    chain = np.zeros((3000, 3), np.float32)
    chain[:, 0] = np.arange(3000, dtype=np.float32) * 0.25
    c.append(("chain 3000 at d", chain, 0.25, 1, big, 0))
    edge = np.array([[8191.999, -8191.999, 0.0], [8191.75, -8191.75, 0.1]], np.float32)
    c.append(("range edge", edge, 0.5, 1, big, 1))
    c.append(("d = 0", f.xyz[:100], 0.0, 1, big, 1))
    c.append(("min > max", f.xyz[:100], 0.3, 10, 5, 1))
    nan = f.xyz[:100].copy()
    nan[37, 1] = np.nan
    c.append(("NaN", nan, 0.3, 1, big, 1))
    far = f.xyz[:100].copy()
    far[3, 2] = 9000.0
    c.append(("out of range", far, 0.3, 1, big, 1))
    return c


@pytest.fixture(scope="module")
def sanitized_exe(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("asan")
    probe = d / "probe.c"
    probe.write_text("int main(void){return 0;}\n")
    r = subprocess.run([gcc, *FLAGS, str(probe), "-o", str(d / "probe")], capture_output=True)
    if r.returncode != 0:
        pytest.skip("this gcc has no address/undefined sanitizer runtime")
    exe = d / "oracle_sanitized"
    r = subprocess.run([gcc, *FLAGS, os.path.join(ROOT, "oracle", "fec_oracle.c"),
                        os.path.join(HERE, "oracle_sanitize_main.c"), "-lm", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe), d


def test_oracle_clean_under_asan_and_ubsan(sanitized_exe):
    exe, d = sanitized_exe
    cases = _cases()
    path = d / "cases.bin"
    with open(path, "wb") as fh:
        for _, xyz, dd, mn, mx, brute in cases:
            xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
            fh.write(struct.pack("<qfqqi", xyz.shape[0], float(dd), int(mn), int(mx), int(brute)))
            fh.write(xyz.tobytes())
    env = dict(os.environ)
    # leak checking needs ptrace-free process inspection, which some
    # containers forbid; invalid accesses and undefined behaviour still abort
    env["ASAN_OPTIONS"] = "detect_leaks=0:abort_on_error=0:exitcode=86"
    env["UBSAN_OPTIONS"] = "print_stacktrace=1:halt_on_error=1:exitcode=87"
    r = subprocess.run([exe, str(path)], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-4000:]
    lines = r.stdout.strip().splitlines()
    assert len(lines) == len(cases)
    for (name, xyz, dd, mn, mx, brute), line in zip(cases, lines):
        parts = line.split()
        st, k, h = int(parts[0]), int(parts[1]), int(parts[2], 16)
        want = oracle.status_of(oracle.cluster, xyz, dd, mn, mx)
        assert (oracle.STATUS_NAMES.get(st) if st else "OK") == want, (name, st, want)
        if st == 0:
            lab, kw = oracle.cluster(xyz, dd, mn, mx)
            assert k == kw and h == _fnv(lab), name
        if brute:
            assert int(parts[3]) == st and int(parts[4]) == 1, (name, line)
