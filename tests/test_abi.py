"""The C ABI: every entry point declared in include/gpubp.h is exported by the built library
(no GPU needed: loading the library and resolving symbols does not touch the device)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "gpubp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_20499_gb300 import build
    try:
        path = build.build()
    except (RuntimeError, FileNotFoundError) as e:
        pytest.skip(f"nvcc unavailable: {e}")
    return ctypes.CDLL(path)


def test_header_parses():
    names = declared()
    for must in ("mip_load_csr", "bp_propagate", "bp_probe_batch", "bp_probe_priority", "probe_split",
                 "probe_cache_apply", "pdhg_solve", "local_search_mtm", "extended_fp", "fix_and_propagate"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_host_only_entry_points(lib):
    lib.bp_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.bp_version()
    box = (ctypes.c_double * 4)()
    lib.probe_split.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    assert lib.probe_split(1, 0.0, 100.0, box) == 1
    assert list(box) == [0.0, 49.0, 50.0, 100.0]
    assert lib.probe_split(0, 0.0, 1.0, box) == 0


def test_no_oracle_in_library(lib):
    """The library must not link or contain the oracle."""
    path = os.path.join(ROOT, "paper_2510_20499_gb300", "libgpubp.so")
    out = subprocess.run(["nm", "-D", path], capture_output=True, text=True).stdout
    assert "orc_" not in out
