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


def test_create_argument_and_flag_checks(libpath):
    """ffs_create_ex rejects bad arguments and unsupported flag combinations before it
    touches the device, with the status codes the header states."""
    import numpy as np

    from paper_2109_07358_gb300 import ffs

    L = ffs.lib()
    U = np.zeros((8, 4))
    p = U.ctypes.data_as(ctypes.c_void_p)
    h = ctypes.c_void_p(1234)
    DF = ffs.FFS_STATE_DF64
    cases = [
        (dict(U=None), ffs.FFS_E_ARG),
        (dict(dtype=7), ffs.FFS_E_ARG),
        (dict(N=0), ffs.FFS_E_ARG),
        (dict(L=3), ffs.FFS_E_ARG),                        # L < N
        (dict(ldU=3), ffs.FFS_E_ARG),                      # ldU < N
        (dict(L=(1 << 30) + 1), ffs.FFS_E_ARG),
        (dict(flags=0x80000), ffs.FFS_E_ARG),              # unknown bit
        (dict(flags=0x30), ffs.FFS_E_ARG),                 # no such state
        (dict(flags=0x300), ffs.FFS_E_ARG),                # no such form
        (dict(flags=0x4), ffs.FFS_E_ARG),                  # no such residual
        (dict(flags=ffs.FFS_FORM_GROUPED | ffs.FFS_RES_FP32), ffs.FFS_E_ARG),
        (dict(flags=ffs.FFS_FORM_GROUPED | ffs.FFS_TAIL_UNBLOCKED), ffs.FFS_E_ARG),
        (dict(flags=ffs.FFS_TAIL_UNBLOCKED | DF), ffs.FFS_E_ARG),
        (dict(flags=ffs.FFS_TRAILING_TC | ffs.FFS_STATE_FP64), ffs.FFS_E_UNSUPPORTED),
        (dict(flags=ffs.FFS_TRAILING_TC | ffs.FFS_STATE_FP32), ffs.FFS_E_UNSUPPORTED),
        (dict(flags=ffs.FFS_TRAILING_TC | DF | ffs.FFS_RES_FP32), ffs.FFS_E_UNSUPPORTED),
        (dict(flags=ffs.FFS_TRAILING_TC | DF | ffs.FFS_TAIL_UNBLOCKED), ffs.FFS_E_UNSUPPORTED),
        (dict(flags=ffs.FFS_TRAILING_TC | DF | ffs.FFS_FORM_PLAIN), ffs.FFS_E_UNSUPPORTED),
    ]
    for kw, want in cases:
        a = dict(U=p, dtype=ffs.FFS_F64, L=8, N=4, ldU=4, flags=0)
        a.update(kw)
        h.value = 1234
        got = L.ffs_create_ex(a["U"], a["dtype"], a["L"], a["N"], a["ldU"], a["flags"], None, ctypes.byref(h))
        assert got == want, (kw, got)
        assert h.value is None                             # *out is cleared on failure
        assert L.ffs_last_error(None).startswith(b"ffs_create_ex")
    assert L.ffs_create_ex(p, ffs.FFS_F64, 8, 4, 4, 0, None, None) == ffs.FFS_E_ARG  # out NULL


def test_noalloc_argument_checks(libpath):
    """ffs_sample_noalloc checks its arguments and the fixed working array's capacity
    before any device call; B = 0 is a no-op."""
    import numpy as np

    from paper_2109_07358_gb300 import ffs

    L = ffs.lib()
    U = np.zeros((8, 4))
    x = np.zeros((4, 4), np.int32)
    p, px = U.ctypes.data_as(ctypes.c_void_p), x.ctypes.data_as(ctypes.c_void_p)
    F64, C128 = ffs.FFS_F64, ffs.FFS_C128
    assert L.ffs_sample_noalloc(p, F64, 8, 4, 0, 0, px, None) == ffs.FFS_OK
    for args in ((None, F64, 8, 4, 4), (p, F64, 8, 4, -1), (p, F64, 8, 0, 4), (p, F64, 3, 4, 4),
                 (p, ffs.FFS_F32, 8, 4, 4), (p, ffs.FFS_C64, 8, 4, 4)):
        assert L.ffs_sample_noalloc(args[0], args[1], args[2], args[3], args[4], 0, px, None) == ffs.FFS_E_ARG
    assert L.ffs_sample_noalloc(p, F64, 8, 4, 4, 0, None, None) == ffs.FFS_E_ARG
    # a working set beyond the fixed array: B (8 N^2 + 4 L + 8 N) bytes and more
    assert L.ffs_sample_noalloc(p, C128, 1 << 20, 64, 4096, 0, px, None) == ffs.FFS_E_NOMEM
    assert b"working memory" in L.ffs_last_error(None)


def test_no_cpu_fallback_without_a_gpu(libpath):
    """On a machine without a usable GPU the product path refuses with FFS_E_CUDA: there
    is no CPU fallback for a sampler or for the allocation-free entry point."""
    import numpy as np
    import torch

    from paper_2109_07358_gb300 import ffs
    from paper_2109_07358_gb300 import workloads as w

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    U = w.haar(16, 4, seed=1, complex_=False)
    with pytest.raises(ffs.FFSError) as e:
        ffs.Sampler(U, 0)
    assert e.value.code == ffs.FFS_E_CUDA
    x = np.zeros((2, 4), np.int32)
    with pytest.raises(ffs.FFSError) as e:
        ffs.ffs_sample_noalloc(U, ffs.FFS_F64, 16, 4, 2, 0, x)
    assert e.value.code == ffs.FFS_E_CUDA
