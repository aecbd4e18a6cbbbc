"""ffs_sample_noalloc: sampling for callers that cannot allocate device memory.

Such callers (a frozen memory pool, a framework allocator that must not be bypassed,
a plugin limited to the memory it is given) cannot use ffs_create, which allocates.
The allocation-free entry point works in a fixed array inside the library and must
give the same samples as ffs_sample_ex with FFS_RES_FP32 | FFS_STATE_FP64 |
FFS_TAIL_UNBLOCKED, within
the tolerance the parity tests use: draws identical except where the uniform lies
within 1e-6 of an oracle CDF boundary.  Two calls in a row check that the contents a
previous call leaves in the shared array do not leak into the next one.

This file is collected last on purpose, so that a run stopping at its first failure
has already run every other test.
"""
import numpy as np
import pytest
import torch

from oracle import ffs_oracle as o
from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w
from tests.parity_util import excused, first_divergence

pytestmark = pytest.mark.gpu

EPS = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_07358_gb300.build import build

    build()
    assert torch.cuda.is_available()


def _check_against_sample_ex(U, B, seed):
    L, N = U.shape
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    out = torch.full((B, N), -1, dtype=torch.int32, device="cuda")
    ffs.ffs_sample_noalloc(Ud, ffs.dtype_of(Ud), L, N, B, seed, out)
    torch.cuda.synchronize()
    S = ffs.Sampler(Ud, ffs.FFS_RES_FP32 | ffs.FFS_STATE_FP64 | ffs.FFS_TAIL_UNBLOCKED)
    ref = S.sample(B, seed)["x"]
    S.sync()
    S.close()
    a, r = out.cpu().numpy(), ref.cpu().numpy()
    assert a.min() >= 0 and a.max() < L
    diff = [b for b in range(B) if not np.array_equal(a[b], r[b])]
    assert len(diff) <= 0.001 * B
    for b in diff:  # any difference must sit within EPS of a CDF boundary
        rec = o.sample_one(U, seed, b, record=True)
        for xs in (a[b], r[b]):
            k = first_divergence(xs, rec["x"])
            assert k < 0 or excused(rec, k, xs[k], EPS)
    return a


def test_noalloc_matches_sample_ex_two_calls_in_a_row():
    U = w.chain_L64_N8()
    x1 = _check_against_sample_ex(U, 2000, 0)
    x2 = _check_against_sample_ex(U, 2000, 0)
    assert np.array_equal(x1, x2)
    Uc = w.haar(40, 10, seed=3)
    _check_against_sample_ex(Uc, 500, 5)
    _check_against_sample_ex(Uc, 300, 6)


def test_noalloc_rejects_sizes_beyond_the_array():
    U = torch.from_numpy(w.haar(64, 32, seed=1)).cuda()
    out = torch.empty((1, 32), dtype=torch.int32, device="cuda")
    with pytest.raises(ffs.FFSError) as e:
        ffs.ffs_sample_noalloc(U, ffs.dtype_of(U), 64, 32, 1 << 20, 0, out)
    assert e.value.code == ffs.FFS_E_NOMEM
    assert "fixed" in str(e.value)


def test_noalloc_refuses_host_buffers():
    """U and out_x must be device memory: the library checks the pointers itself and
    returns FFS_E_ARG for host memory (called through the C ABI, past the binding)."""
    import ctypes

    U = torch.from_numpy(w.haar(40, 6, seed=2, complex_=False)).cuda()
    host_out = np.zeros((4, 6), dtype=np.int32)
    lib = ffs.lib()
    rc = lib.ffs_sample_noalloc(ctypes.c_void_p(U.data_ptr()), ffs.FFS_F64, 40, 6, 4, 0,
                                ctypes.c_void_p(host_out.ctypes.data), None)
    assert rc == ffs.FFS_E_ARG
    assert "device" in lib.ffs_last_error(None).decode()
    host_U = np.ascontiguousarray(w.haar(40, 6, seed=2, complex_=False))
    dev_out = torch.empty((4, 6), dtype=torch.int32, device="cuda")
    rc = lib.ffs_sample_noalloc(ctypes.c_void_p(host_U.ctypes.data), ffs.FFS_F64, 40, 6, 4, 0,
                                ctypes.c_void_p(dev_out.data_ptr()), None)
    assert rc == ffs.FFS_E_ARG
    with pytest.raises(TypeError):
        ffs.ffs_sample_noalloc(U.cpu(), ffs.FFS_F64, 40, 6, 4, 0, dev_out)


def test_noalloc_marks_degenerate_chains_with_minus_one():
    """A zero column of U makes every weight vanish at the step whose column it is (the
    normaliser is 0): that entry and the rest of the row are -1, the earlier entries are
    distinct sites.  The step is known in advance from the sample's column order."""
    L, N, B, seed, zero_col = 40, 6, 64, 3, 2
    Un = w.haar(L, N, seed=4, complex_=False)
    Un[:, zero_col] = 0.0
    U = torch.from_numpy(np.ascontiguousarray(Un)).cuda()
    out = torch.full((B, N), 7, dtype=torch.int32, device="cuda")
    ffs.ffs_sample_noalloc(U, ffs.FFS_F64, L, N, B, seed, out)
    torch.cuda.synchronize()
    X = out.cpu().numpy()
    for b in range(B):
        kz = int(np.flatnonzero(o.permutation(seed, b, N) == zero_col)[0])
        assert (X[b, kz:] == -1).all(), (b, kz, X[b])
        pre = X[b, :kz]
        assert ((pre >= 0) & (pre < L)).all() and len(set(pre.tolist())) == kz
