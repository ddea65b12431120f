"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/fec.h declares; host-only entry points work without a GPU;
the binding fails loudly without the library."""
import os
import re

import pytest

from paper_2208_07678_gb300 import build as libbuild
from paper_2208_07678_gb300 import fec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fec_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return fec.load()


def test_every_declared_symbol_is_exported(lib):
    import ctypes

    declared = header_functions()
    assert declared >= set(fec.EXPORTS)
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_exports_match_nm(lib):
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", libbuild.LIB], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (fec_[a-z_0-9]+)", out))
    assert header_functions() <= exported


def test_debug_build_exports_the_same_functions():
    """The bounds-checked debug library (-DFEC_DEBUG=1) builds and exports
    every declared function, like the release library."""
    import subprocess

    path = libbuild.build(debug=True)
    assert path == libbuild.LIB_DEBUG and os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    assert header_functions() <= set(re.findall(r"\bT (fec_[a-z_0-9]+)", out))


def test_status_strings(lib):
    for code, name in fec.STATUS.items():
        assert fec.fec_status_string(code) == name


def test_workspace_bytes_host_only(lib):
    a = fec.fec_workspace_bytes(1000, 0.5)
    b = fec.fec_workspace_bytes(1_000_000, 0.5)
    assert 0 < a < b
    assert fec.fec_workspace_bytes(-1, 0.5) == -1
    assert fec.fec_workspace_bytes(10, 0.0) == -1
    assert 100 < b / 1_000_000 < 500  # bytes per point of the device workspace


def test_create_without_gpu_reports_cuda_error(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("host has a GPU")
    with pytest.raises(fec.FecError) as e:
        fec.fec_create(0)
    assert e.value.name == "FEC_ERR_CUDA"


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(fec, "_lib", None)
    monkeypatch.setattr(libbuild, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        fec.load()


def test_product_path_does_not_import_oracle():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2208_07678_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "fec_oracle" not in src, f


def test_library_selection_by_environment(monkeypatch):
    """FEC_LIBRARY=debug selects the bounds-checked build; anything else the release one."""
    monkeypatch.setenv("FEC_LIBRARY", "debug")
    assert fec.debug_library() and fec.library_path() == libbuild.LIB_DEBUG
    monkeypatch.setenv("FEC_LIBRARY", "release")
    assert not fec.debug_library() and fec.library_path() == libbuild.LIB
    monkeypatch.delenv("FEC_LIBRARY")
    assert fec.library_path() == libbuild.LIB
