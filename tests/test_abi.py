"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares (no GPU needed; no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ffs_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2109_07358_gb300.build import build

    return build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ffs_create", "ffs_create_ex", "ffs_sample", "ffs_sample_ex", "ffs_sync", "ffs_last_error",
              "ffs_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_2109_07358_gb300 import ffs

    monkeypatch.setattr(ffs, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(ffs, "_lib", None)
    with pytest.raises(RuntimeError):
        ffs.lib()


def test_null_handle_calls_fail_cleanly(libpath):
    from paper_2109_07358_gb300 import ffs

    L = ffs.lib()
    assert L.ffs_sync(None) == ffs.FFS_E_ARG
    assert L.ffs_sample(None, 1, 0, None) == ffs.FFS_E_ARG
    assert b"NULL" in L.ffs_last_error(None)
    L.ffs_destroy(None)
