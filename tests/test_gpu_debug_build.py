"""The bounds-checked debug build (libfec_debug.so, -DFEC_DEBUG=1) on the GPU.

Debug builds check the indices of the gathers and scatters that depend on
device-computed offsets (sorted positions, sub-cell and cell numbers, region
indices, neighbour tables, queued pairs, parent chains, ranks, labels); a
failed check ends the call with FEC_ERR_INTERNAL instead of touching memory
out of bounds.  Here the core parity suites run again in a child process with
FEC_LIBRARY=debug: every case must still equal the oracle exactly, with no
check failing, and the child must have loaded the debug library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SUITES = ["test_gpu_parity.py", "test_gpu_failure.py", "test_gpu_batch_segments.py"]


@pytest.fixture(scope="module")
def debug_env():
    from paper_2208_07678_gb300 import build as libbuild

    libbuild.build()
    libbuild.build(debug=True)
    env = dict(os.environ)
    env["FEC_LIBRARY"] = "debug"
    return env


def test_debug_library_is_the_one_loaded(debug_env):
    code = (
        "import numpy as np, torch\n"
        "from paper_2208_07678_gb300 import fec, synth\n"
        "c = synth.blobs_20k()\n"
        "with fec.Context(device=0) as ctx:\n"
        "    lab, k = ctx.cluster(c.xyz, c.d, c.min_size, c.max_size)\n"
        "maps = open('/proc/self/maps').read()\n"
        "print('debug' if 'libfec_debug.so' in maps and 'libfec.so' not in maps else 'release', k)\n"
    )
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=debug_env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    kind, k = r.stdout.split()
    assert kind == "debug" and int(k) > 0


def test_parity_suites_under_bounds_checks(debug_env):
    cmd = [sys.executable, "-m", "pytest", *[os.path.join(HERE, s) for s in SUITES], "-m", "gpu",
           "-x", "-q", "-p", "no:cacheprovider"]
    r = subprocess.run(cmd, cwd=ROOT, env=debug_env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, (r.stdout[-4000:], r.stderr[-2000:])
    assert " passed" in r.stdout
