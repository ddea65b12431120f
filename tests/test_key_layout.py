"""The grid-key layout of the CUDA library, checked on the CPU.

``tests/key_layout_main.cu`` includes the library's internal header and runs
its key-layout code (the bricked cell key: encode, decode, column and slab
keys; the per-point sort key and its unpacking) on the host: round trips for
random bit widths, axis orders and coordinates (32- and 64-bit keys), and an
exhaustive bijection check for small widths.  It is compiled with nvcc for
the host only and needs no GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_key_layout_round_trips(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "key_layout"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-I",
                        os.path.join(ROOT, "include"), "-I",
                        os.path.join(ROOT, "paper_2208_07678_gb300", "csrc"),
                        os.path.join(HERE, "key_layout_main.cu"), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "failures=0" in r.stdout
