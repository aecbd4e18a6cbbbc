"""Python binding of libffs (ctypes).  Argument marshalling only: every step of the
sampler runs in the CUDA library; nothing here computes.

Functions carry the names of the C entry points declared in include/ffs.h.  Array
arguments may be torch tensors (host or device), numpy arrays, or raw integer
addresses; they are passed as pointers.  A non-zero status raises FFSError.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libffs.so")

# Status codes, dtypes and flags (mirrors include/ffs.h).
FFS_OK = 0
FFS_E_ARG = 1
FFS_E_NOT_ORTHONORMAL = 2
FFS_E_NOMEM = 3
FFS_E_CUDA = 4
FFS_E_NUMERIC = 5
FFS_E_TIMEOUT = 6
FFS_E_BUSY = 7
FFS_E_UNSUPPORTED = 8
FFS_F64, FFS_C128, FFS_F32, FFS_C64 = 0, 1, 2, 3
FFS_RES_BF16X3 = 0x0
FFS_RES_FP32 = 0x1
FFS_RES_BF16 = 0x2
FFS_RES_TF32 = 0x3
FFS_STATE_FP64 = 0x00
FFS_STATE_FP32 = 0x10
FFS_STATE_DF64 = 0x20
FFS_FORM_BATCHED = 0x000
FFS_FORM_PLAIN = 0x100
FFS_FORM_GROUPED = 0x200
FFS_GROUP_SIZE = 128
FFS_NO_ORTHO_CHECK = 0x1000
FFS_TAIL_UNBLOCKED = 0x2000
FFS_TRAILING_TC = 0x4000
FFS_FAULT_NONE, FFS_FAULT_SKIP_ARRIVAL = 0, 1

_lib = None


class FFSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[ffs status {code}] {msg}")
        self.code = code


class ffs_csr(ctypes.Structure):
    """Sparse n x n matrix in CSR form; every array is device memory."""
    _fields_ = [("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("nnz", ctypes.c_int64)]


def lib() -> ctypes.CDLL:
    """Load libffs.so (built in-tree).  Raises when it is missing: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run paper_2109_07358_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, u64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
        L.ffs_create.argtypes = [vp, i64, i64, ctypes.POINTER(vp)]
        L.ffs_create_ex.argtypes = [vp, i32, i64, i64, i64, ctypes.c_uint, vp, ctypes.POINTER(vp)]
        L.ffs_sample.argtypes = [vp, i64, u64, vp]
        L.ffs_sample_ex.argtypes = [vp, i64, u64, u64, i64, vp, vp, vp, vp, vp, vp]
        L.ffs_sync.argtypes = [vp]
        L.ffs_last_error.argtypes = [vp]
        L.ffs_last_error.restype = ctypes.c_char_p
        L.ffs_destroy.argtypes = [vp]
        L.ffs_destroy.restype = None
        L.ffs_query.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                ctypes.POINTER(ctypes.c_uint), i64, ctypes.POINTER(i64)]
        L.ffs_sample_noalloc.argtypes = [vp, i32, i64, i64, i64, u64, vp, vp]
        L.ffs_sample_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(u64),
                                         ctypes.POINTER(vp), i32, vp]
        L.ffs_server_create.argtypes = [ctypes.c_size_t, ctypes.c_uint, i32, vp, ctypes.POINTER(vp)]
        L.ffs_submit.argtypes = [vp, vp, i32, i64, i64, i64, u64, vp, ctypes.POINTER(u64)]
        L.ffs_wait.argtypes = [vp, u64, i32, ctypes.POINTER(ctypes.c_double)]
        L.ffs_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                       ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(i64)]
        L.ffs_server_destroy.argtypes = [vp]
        L.ffs_server_destroy.restype = None
        L.ffs_profile.argtypes = [vp, i32]
        L.ffs_debug_inject.argtypes = [vp, i32]
        L.ffs_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), i32]
        L.ffs_sample_metropolis.argtypes = [vp, i64, u64, u64, i64, i64, vp, vp, vp]
        L.ffs_sample_lensemble.argtypes = [vp, vp, i64, u64, u64, vp, vp, vp, vp, vp, vp, vp]
        L.ffs_jastrow_estimate.argtypes = [vp, i64, i64, i64, ctypes.POINTER(ffs_csr), vp, ctypes.POINTER(ffs_csr),
                                           vp, vp, vp, vp]
        for name in ("ffs_create", "ffs_create_ex", "ffs_sample", "ffs_sample_ex", "ffs_sync", "ffs_query",
                     "ffs_profile", "ffs_profile_read", "ffs_sample_noalloc", "ffs_sample_batched",
                     "ffs_server_create", "ffs_submit", "ffs_wait", "ffs_server_stats", "ffs_jastrow_estimate",
                     "ffs_sample_lensemble", "ffs_sample_metropolis", "ffs_debug_inject"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _ptr(obj):
    if obj is None:
        return None
    if isinstance(obj, int):
        return ctypes.c_void_p(obj)
    if hasattr(obj, "data_ptr"):
        return ctypes.c_void_p(obj.data_ptr())
    if hasattr(obj, "ctypes"):
        return ctypes.c_void_p(obj.ctypes.data)
    raise TypeError(f"cannot pass {type(obj)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(s.cuda_stream)  # torch.cuda.Stream


def _check(code: int, handle=None):
    if code != FFS_OK:
        msg = lib().ffs_last_error(handle)
        raise FFSError(code, msg.decode() if msg else "")


def ffs_create(U, L: int, N: int):
    h = ctypes.c_void_p()
    _check(lib().ffs_create(_ptr(U), L, N, ctypes.byref(h)))
    return h


def ffs_create_ex(U, dtype: int, L: int, N: int, ldU: int, flags: int = 0, stream=None):
    h = ctypes.c_void_p()
    _check(lib().ffs_create_ex(_ptr(U), dtype, L, N, ldU, flags, _stream(stream), ctypes.byref(h)))
    return h


def ffs_sample(h, B: int, seed: int, out_x):
    _check(lib().ffs_sample(h, B, seed, _ptr(out_x)), h)


def ffs_sample_ex(h, B: int, seed: int, first_sample_index: int, n_steps: int, out_x, out_perm=None,
                  out_logp=None, force_x=None, out_probs=None, stream=None):
    _check(lib().ffs_sample_ex(h, B, seed, first_sample_index, n_steps, _ptr(out_x), _ptr(out_perm),
                               _ptr(out_logp), _ptr(force_x), _ptr(out_probs), _stream(stream)), h)


def ffs_sample_lensemble(h, lam, B: int, seed: int, first_sample_index: int, out_x, out_n=None, out_perm=None,
                         out_logp=None, force_x=None, out_probs=None, stream=None):
    _check(lib().ffs_sample_lensemble(h, _ptr(lam), B, seed, first_sample_index, _ptr(out_x), _ptr(out_n),
                                      _ptr(out_perm), _ptr(out_logp), _ptr(force_x), _ptr(out_probs),
                                      _stream(stream)), h)


def ffs_sample_metropolis(h, B: int, seed: int, first_sample_index: int, n_steps: int, m_cond: int, out_x,
                          out_perm=None, stream=None):
    _check(lib().ffs_sample_metropolis(h, B, seed, first_sample_index, n_steps, m_cond, _ptr(out_x),
                                       _ptr(out_perm), _stream(stream)), h)


def ffs_sample_noalloc(U, dtype: int, L: int, N: int, B: int, seed: int, out_x, stream=None):
    """Sampling that allocates no device memory (fixed working array in the library);
    for callers that cannot allocate.  U and out_x must be device memory; a row of
    out_x that holds -1 from some step on is a sample whose chain became degenerate."""
    for name, t in (("U", U), ("out_x", out_x)):
        if hasattr(t, "is_cuda") and not t.is_cuda:
            raise TypeError(f"ffs_sample_noalloc: {name} must be a CUDA tensor")
    _check(lib().ffs_sample_noalloc(_ptr(U), dtype, L, N, B, seed, _ptr(out_x), _stream(stream)))


def ffs_sample_batched(handles, Bs, seeds, outs, stream=None):
    """Sample many instances together (one grouped, graph-captured schedule)."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    b = (ctypes.c_int64 * n)(*Bs)
    sd = (ctypes.c_uint64 * n)(*seeds)
    o = (ctypes.c_void_p * n)(*[_ptr(x).value if x is not None else None for x in outs])
    _check(lib().ffs_sample_batched(hs, b, sd, o, n, _stream(stream)), handles[0])


def ffs_server_create(hbm_budget: int = 0, flags: int = 0, max_active: int = 0, stream=None):
    s = ctypes.c_void_p()
    _check(lib().ffs_server_create(hbm_budget, flags, max_active, _stream(stream), ctypes.byref(s)))
    return s


def ffs_submit(server, U, dtype: int, L: int, N: int, n_samples: int, seed: int, out_x) -> int:
    rid = ctypes.c_uint64()
    _check(lib().ffs_submit(server, _ptr(U), dtype, L, N, n_samples, seed, _ptr(out_x), ctypes.byref(rid)))
    return rid.value


def ffs_wait(server, req_id: int, timeout_ms: int = -1) -> float:
    """Block until the request is done; returns its latency in ms (submission to completion)."""
    lat = ctypes.c_double()
    _check(lib().ffs_wait(server, req_id, timeout_ms, ctypes.byref(lat)))
    return lat.value


def ffs_server_stats(server):
    p, a, it, b, pk = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t(), ctypes.c_int64()
    _check(lib().ffs_server_stats(server, ctypes.byref(p), ctypes.byref(a), ctypes.byref(it), ctypes.byref(b),
                                  ctypes.byref(pk)))
    return {"pending": p.value, "active": a.value, "iterations": it.value, "bytes_in_use": b.value,
            "peak_active": pk.value}


def ffs_server_destroy(server):
    lib().ffs_server_destroy(server)


def ffs_debug_inject(h, fault: int):
    """Failure-path testing: arm a one-shot fault for the next tensor-core residual launch."""
    _check(lib().ffs_debug_inject(h, fault), h)


def ffs_sync(h):
    _check(lib().ffs_sync(h), h)


def ffs_last_error(h=None) -> str:
    msg = lib().ffs_last_error(h)
    return msg.decode() if msg else ""


def ffs_destroy(h):
    lib().ffs_destroy(h)


def ffs_query(h, B: int = 0):
    L, N, bts = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    dt, fl = ctypes.c_int(), ctypes.c_uint()
    _check(lib().ffs_query(h, ctypes.byref(L), ctypes.byref(N), ctypes.byref(dt), ctypes.byref(fl), B,
                           ctypes.byref(bts)), h)
    return {"L": L.value, "N": N.value, "dtype": dt.value, "flags": fl.value, "bytes_for_B": bts.value}


FFS_PHASE_PERM, FFS_PHASE_RESIDUAL, FFS_PHASE_TAIL, FFS_PHASE_PANEL, FFS_PHASE_PANEL_S = 0, 1, 2, 3, 4
FFS_PHASE_PANEL_TC = 5
FFS_NUM_PHASES = 6
PHASE_NAMES = ("perm", "residual", "tail", "panel", "panel_s", "panel_tc")


def ffs_profile(h, enable: bool = True):
    _check(lib().ffs_profile(h, 1 if enable else 0), h)


def ffs_profile_read(h):
    """{phase name: (total device ms, launches)} since profiling was enabled."""
    ms = (ctypes.c_double * FFS_NUM_PHASES)()
    n = (ctypes.c_int64 * FFS_NUM_PHASES)()
    _check(lib().ffs_profile_read(h, ms, n, FFS_NUM_PHASES), h)
    return {PHASE_NAMES[p]: (ms[p], n[p]) for p in range(FFS_NUM_PHASES)}


def _csr(m):
    if m is None:
        return None
    rowptr, col, val = m
    return ctypes.byref(ffs_csr(rowptr.data_ptr(), col.data_ptr(), val.data_ptr(), int(val.numel())))


def ffs_jastrow_estimate(x, n_orb: int, v=None, o=None, q=None, out_logj2=None, out_obs=None, stream=None):
    """Reweighting estimate of a diagonal observable in the Jastrow state J |phi_0> from the
    free-fermion samples x (device int32 tensor, B x n_occ).  v and q are (rowptr int64,
    col int32, val float64) device tensors or None, o a float64 device tensor or None.
    Returns {"mean", "log_j2_mean", "ess", "stderr"}."""
    B, n_occ = int(x.shape[0]), int(x.shape[1])
    res = (ctypes.c_double * 4)()
    _check(lib().ffs_jastrow_estimate(_ptr(x), B, n_occ, int(n_orb), _csr(v), _ptr(o), _csr(q), _ptr(out_logj2),
                                      _ptr(out_obs), ctypes.cast(res, ctypes.c_void_p), _stream(stream)))
    return {"mean": res[0], "log_j2_mean": res[1], "ess": res[2], "stderr": res[3]}


def dtype_of(U) -> int:
    """FFS dtype code of a torch tensor or numpy array."""
    name = str(U.dtype).replace("torch.", "")
    return {"float64": FFS_F64, "complex128": FFS_C128, "float32": FFS_F32, "complex64": FFS_C64}[name]


class Sampler:
    """Owns one handle: ``Sampler(U, flags).sample(B, seed)`` -> torch int32 (B, N) on U's device."""

    def __init__(self, U, flags: int = 0, stream=None):
        self.L, self.N = int(U.shape[0]), int(U.shape[1])
        if stream is not None and getattr(U, "is_cuda", False):
            import torch

            stream.wait_stream(torch.cuda.current_stream())  # U must be ready on the handle's stream
        self.h = ffs_create_ex(U, dtype_of(U), self.L, self.N, int(U.stride(0)) if hasattr(U, "stride")
                               else self.N, flags, stream)

    def sample(self, B: int, seed: int = 0, first_sample_index: int = 0, n_steps: int = 0, out=None,
               device="cuda", perm=False, logp=False, force_x=None, probs=False, stream=None):
        import torch

        K = n_steps or self.N
        x = out if out is not None else torch.empty((B, K), dtype=torch.int32, device=device)
        pm = torch.empty((B, self.N), dtype=torch.int32, device=device) if perm else None
        lp = torch.empty((B,), dtype=torch.float64, device=device) if logp else None
        pr = torch.empty((B, K, self.L), dtype=torch.float32, device=device) if probs else None
        ffs_sample_ex(self.h, B, seed, first_sample_index, n_steps, x, pm, lp, force_x, pr, stream)
        res = {"x": x}
        if perm:
            res["perm"] = pm
        if logp:
            res["logp"] = lp
        if probs:
            res["probs"] = pr
        return res

    def sample_lensemble(self, lam, B: int, seed: int = 0, first_sample_index: int = 0, perm=False, logp=False,
                         force_x=None, probs=False, stream=None, device="cuda"):
        """L-ensemble draws with eigenvalues lam (one per column of U): dict with 'x' (B x N,
        -1 past each sample's n_b), 'n' (B), and the optional outputs."""
        import torch

        x = torch.empty((B, self.N), dtype=torch.int32, device=device)
        n = torch.empty((B,), dtype=torch.int32, device=device)
        pm = torch.empty((B, self.N), dtype=torch.int32, device=device) if perm else None
        lp = torch.empty((B,), dtype=torch.float64, device=device) if logp else None
        pr = torch.empty((B, self.N, self.L), dtype=torch.float32, device=device) if probs else None
        ffs_sample_lensemble(self.h, lam, B, seed, first_sample_index, x, n, pm, lp, force_x, pr, stream)
        res = {"x": x, "n": n}
        if perm:
            res["perm"] = pm
        if logp:
            res["logp"] = lp
        if probs:
            res["probs"] = pr
        return res

    def sample_metropolis(self, B: int, m_cond: int, seed: int = 0, first_sample_index: int = 0, n_steps: int = 0,
                          perm=False, stream=None, device="cuda"):
        """Large-L draws (Metropolis chain of m_cond updates per step): dict with 'x'
        (B x n_steps) and optionally 'perm'."""
        import torch

        K = n_steps or self.N
        x = torch.empty((B, K), dtype=torch.int32, device=device)
        pm = torch.empty((B, self.N), dtype=torch.int32, device=device) if perm else None
        ffs_sample_metropolis(self.h, B, seed, first_sample_index, n_steps, m_cond, x, pm, stream)
        res = {"x": x}
        if perm:
            res["perm"] = pm
        return res

    def sync(self):
        ffs_sync(self.h)

    def close(self):
        if self.h is not None:
            ffs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
