#!/usr/bin/env python
"""Benchmark of the fast-fermion-sampling hot path (arXiv 2109.07358) on GB300.

A step is one ffs_sample call: the whole chain (permutations, N residual steps, N
draw + state-update steps) over one batch of B samples of the workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ffs|reference]

Default workload: the largest configuration, a 1D open Anderson chain L = 16384 with
on-site disorder U[-1, 1] (seed 0), the N = 2048 lowest orbitals (real), B = 8192
samples, Philox seed 0.  Prints one JSON line (rank 0).  Under torchrun each rank
samples its own index range (weak scaling, no collective on the data path).  Each
timed step has its own CUDA events (their sum is the step time; p50/p99 per call come
from them); a workload whose working set fits in L2 gets the cache flushed between
steps, outside the events.  `roofline` is the residual (GEMM) phase against the
tensor-core peak of its precision; `roofline_tail` is the state update's dominant
kernel.  Further sections: the plain per-sample FP32 form, the CPU oracle, end to end
through host buffers, the 64 x 64 lattice workload (and its IEEE FP64 state), per-call
latency of the L = 64 chain over 200 calls, marginal sampling, the L-ensemble, the
grouped form, the large-L variant, reweighting, batching and a serving-rate sweep.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "lattice64x64_N1024_B4096": dict(
        make="lattice", B=4096, L=4096, N=1024, cplx=True, grid=(64, 64),
        desc="64x64 open square lattice, random U(1) hopping phases (seed 0), N=1024 lowest orbitals, "
             "complex, B=4096 samples, Philox seed 0"),
    "lattice32x32_N256_B1024": dict(
        make="lattice32", B=1024, L=1024, N=256, cplx=True, grid=(32, 32),
        desc="32x32 open square lattice, random U(1) hopping phases (seed 0), N=256 lowest orbitals, "
             "complex, B=1024 samples, Philox seed 0 (reduced case for profiler captures)"),
    "lattice32x32_N256_B4096": dict(
        make="lattice32", B=4096, L=1024, N=256, cplx=True, grid=(32, 32),
        desc="32x32 open square lattice, random U(1) hopping phases (seed 0), N=256 lowest orbitals, "
             "complex, B=4096 samples, Philox seed 0 (a full 4096-sample wave at a size profilers can "
             "replay)"),
    "anderson_L16384_N2048_B8192": dict(
        make="anderson", B=8192, L=16384, N=2048, cplx=False, grid=(1, 16384),
        desc="1D open Anderson chain L=16384, on-site disorder U[-1, 1] (seed 0), N=2048 lowest orbitals, "
             "real, B=8192 samples, Philox seed 0 (the precision workload; the per-sample double-float "
             "state is 16.8 MB in triangular slabs, so the whole batch runs in one wave)"),
    "anderson_L4096_N512_B2048": dict(
        make="anderson4k", B=2048, L=4096, N=512, cplx=False, grid=(1, 4096),
        desc="1D open Anderson chain L=4096, on-site disorder U[-1, 1] (seed 0), N=512 lowest orbitals, real, "
             "B=2048 samples, Philox seed 0 (reduced case for profiler captures)"),
    "chain64_N8_B10000": dict(
        make="chain", B=10000, L=64, N=8, cplx=False, grid=(1, 64),
        desc="1D open chain L=64, N=8 (closed-form orbitals), B=10^4 samples, Philox seed 0"),
}

# Peak denominators (GB300).  FP64 and FP32 CUDA-core rates: nominal unit counts x
# clock (FP64: 1.25 TFLOP/s dense nominal; FP32: 152 SMs x 128 lanes x 2 flops x 2.07 GHz).
NOMINAL_FP64_TFLOPS = 1.25
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
L2_BYTES = 129 * 2**20


def working_set_bytes(L, N, B, cplx, state):
    """Bytes one step touches: the per-sample blocked state (slab s of 32 columns holds
    32 (s + 1) rows: 512 S (S + 1) entries for S = ceil(N / 32) slabs), U in FP64 and its
    BF16 hi/lo copies, the output rows."""
    entry = {"df64": 8, "fp64": 8, "fp32": 4}[state] * (2 if cplx else 1)
    S = (N + 31) // 32
    u = L * N * (2 if cplx else 1) * (8 + 4)
    return B * 512 * S * (S + 1) * entry + u + B * N * 4


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"],
                    source="measured")
    return dict(hbm_gbs=6800.0, bf16=1900.0, bf16_sus=1700.0, source="fallback")


def make_U(spec):
    from paper_2109_07358_gb300 import workloads as w

    if spec["make"] == "lattice":
        return w.lattice_64x64_N1024(0)
    if spec["make"] == "lattice32":
        return w.square_lattice(32, 32, 256, 0)
    if spec["make"] == "chain":
        return w.chain_L64_N8()
    if spec["make"] == "anderson":
        return w.anderson_L16384_N2048(0)
    if spec["make"] == "anderson4k":
        return w.anderson_chain(4096, 512, 1.0, 0)
    raise ValueError(spec["make"])


def flops_per_sample(L, N, cplx):
    """Algorithmic residual flops per sample: the paper's 2Lk per step summed over
    k = 1..N, i.e. L N (N+1) real flops (x4 for complex arithmetic)."""
    return L * N * (N + 1) * (4 if cplx else 1)


def tail_flops_per_sample(N, cplx):
    """Arithmetic of the per-sample Gauss-Jordan state update (unblocked count): at step k
    (0-based, k < N-1) a k x (N-k) product of the new row with the state and a
    k x (N-k-1) rank-1 update, 2 real flops per real multiply-add (8 per complex)."""
    k = np.arange(N - 1, dtype=np.float64)
    macs = float(np.sum(k * (N - k) + k * (N - k - 1)))
    return macs * (8 if cplx else 2)


def blocked_flops_per_sample(N, cplx, nb=32):
    """Algorithmic flops per sample of each kernel of the blocked state update, as the
    kernels compute it (2 real flops per real multiply-add, 8 per complex):
      step     at step k in panel [k0, k1): the new row against the state on the panel
               columns (k x (k1 - k)) and the rank-1 update (k x (k1 - k - 1));
      panel_s  per panel with trailing columns: S = D - C W0_P (nb x k0 x nb) and its
               Gauss-Jordan inverse (nb x nb x 2 nb);
      panel    per panel, T = [k1, N): Y = U - C W0_T (nb x k0 x |T|), S^-1 Y
               (nb x nb x |T|), W0_T - W0_P Bot (k0 x nb x |T|);
      top      the last of these alone (the part the tensor-core trailing update takes)."""
    f = 8 if cplx else 2
    step = panel_s = panel = top = 0.0
    for k in range(N - 1):
        k0 = (k // nb) * nb
        k1 = min(k0 + nb, N)
        step += k * (k1 - k) + k * (k1 - k - 1)
    for k0 in range(0, N, nb):
        k1 = min(k0 + nb, N)
        if k1 >= N:
            break
        T = N - k1
        panel_s += nb * k0 * nb + nb * nb * 2 * nb
        panel += T * nb * (2 * k0 + nb)
        top += T * nb * k0
    return {"step": step * f, "panel_s": panel_s * f, "panel": panel * f, "top": top * f}


def blocked_bytes_per_sample(L, N, e, nb=32, gsum=0):
    """Algorithmic HBM bytes per sample of the memory-bound kernels of the blocked state
    update (e = bytes per state entry: 8 for real double-float or FP64, 16 for complex):
      step  per step k: what the draw reads (the L FP32 weights, or with gsum > 0 the
            residual's sums over groups of gsum sites and the chosen group's weights);
            the live panel block read (k x (k1 - k) entries) and written back
            (k x (k1 - k - 1)); at the first step of a panel the k0 x nb copy W0_P written;
      new   per panel, T = [k1, N): W0_T read (k0 x |T|), the new rows' U entries read and
            the new rows written (2 x nb x |T|);
      top   per panel: W0_T read and Top written (2 x k0 x |T|), W0_P read (k0 x nb)."""
    step = new = top = 0.0
    for k in range(N):
        k0 = (k // nb) * nb
        k1 = min(k0 + nb, N)
        step += 4.0 * ((L + gsum - 1) // gsum + gsum) if gsum else 4.0 * L
        if k + 1 < N:
            step += e * (k * (k1 - k) + k * (k1 - k - 1) + (k0 * nb if k == k0 else 0))
    for k0 in range(0, N, nb):
        k1 = min(k0 + nb, N)
        if k1 >= N:
            break
        T = N - k1
        new += e * (k0 * T + 2 * nb * T)
        top += e * (2 * k0 * T + k0 * nb)
    return {"step": step, "new": new, "top": top}


# Instruction counts behind the derived CUDA-core peaks of the double-float state kernels:
# a real lazy multiply-add (lz_mac) is 13 FP32-pipe instructions for 2 flops; a complex
# one by Karatsuba is three of them (39 instructions) for 8 flops.
DF_INSTR_REAL, DF_INSTR_COMPLEX = 13, 39
FP32_INSTR_PER_S = 152 * 128 * 2.07e9   # FP32 lanes x max clock (nominal)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------------------ CPU oracle
def oracle_baseline(U, n_samples, seed=0, workers=None, threads=1):
    """Time the CPU oracle (as it stands) on n_samples of the workload: one
    single-threaded worker process per core (threads = 1), or one process whose BLAS
    calls use `threads` threads (large workloads, where one sample is tens of seconds on
    one core).  Returns (samples/s, wall seconds, cores used)."""
    if threads > 1:
        workers, blas = 1, str(threads)
    else:
        workers, blas = max(1, min(workers or os.cpu_count() or 1, n_samples)), "1"
    bounds = np.linspace(0, n_samples, workers + 1).astype(int)
    jobs = [(U, seed, int(bounds[i]), int(bounds[i + 1])) for i in range(workers)]
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in saved:  # children read these at their numpy import
        os.environ[v] = blas
    try:
        rate, wall, _ = _oracle_pool(jobs, workers, n_samples, threads)
        return rate, wall, max(workers, threads)
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old


def oracle_plan(U, B, target_s=10.0):
    """(samples, BLAS threads) for a bounded oracle timing of about target_s of wall time.
    Small workloads: one single-threaded worker per core, sized from a probe of one sample
    per core.  Large ones (L N^2, x4 complex, above 1e9 multiply-adds, tens of seconds per
    sample on one core): one process with BLAS on every core, whole samples, at least one."""
    L, N = U.shape
    cores = os.cpu_count() or 1
    if L * N * N * (4 if np.iscomplexobj(U) else 1) <= 1e9:
        n0 = max(2, cores)
        rate, _, _ = oracle_baseline(U, n0)
        return int(min(max(n0, rate * target_s), max(n0, B))), 1
    rate, _, _ = oracle_baseline(U, 1, threads=cores)
    return int(min(B, max(1, round(rate * target_s)))), cores


def _oracle_worker(args):
    U, seed, lo, hi, threads = args
    from oracle import ffs_oracle as o

    if threads == 1:
        o._single_thread()
    t = time.perf_counter()
    for s in range(lo, hi):
        o.sample_one(U, seed, s)
    return time.perf_counter() - t


def _oracle_pool(jobs, workers, n_samples, threads=1):
    import multiprocessing as mp

    U = jobs[0][0]
    jobs = [j + (threads,) for j in jobs]
    with mp.get_context("spawn").Pool(workers) as pool:
        warm = np.linalg.qr(np.random.default_rng(0).standard_normal((8, 2)))[0]  # imports, first BLAS calls
        pool.map(_oracle_worker, [(warm, 0, 0, 1, threads)] * workers)
        t0 = time.perf_counter()
        pool.map(_oracle_worker, jobs)
        wall = time.perf_counter() - t0
    return n_samples / wall, wall, workers


def run_reference(args, spec, rank, world):
    """--impl reference: the CPU oracle on the host cores, same metric and workload."""
    if rank != 0:
        return 0
    U = make_U(spec)
    n, threads = oracle_plan(U, spec["B"])
    if args.ref_samples:
        n = args.ref_samples
    for _ in range(args.warmup):
        oracle_baseline(U, max(1, n // 4), threads=threads)
    rates = []
    walls = []
    for _ in range(args.steps):
        r, wall, workers = oracle_baseline(U, n, threads=threads)
        rates.append(r)
        walls.append(wall)
    v = float(np.median(rates))
    out = {
        "impl": "reference", "metric": "FFS samples/s", "value": v, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.median(walls)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": spec["desc"], "B_per_step": n,
                   "sample": f"{n} samples of the workload per step (indices 0..{n - 1})"},
        "cpu_baseline": {"value": v, "unit": "samples/s", "cores": workers, "kind": "oracle",
                         "sample": f"{n} samples per step, " + ("one single-threaded worker per core" if threads == 1
                                                                 else f"one process, BLAS on {threads} threads")},
        "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------------------ patterns
def bench_batching(args, flags, stream):
    """Many independent instances (Haar U, L log-uniform in [256, 8192], N log-uniform in
    [16, min(1024, L/4)], 64 samples each): one grouped, graph-captured schedule against
    the same instances sampled one after another."""
    import torch

    from paper_2109_07358_gb300 import ffs
    from paper_2109_07358_gb300 import workloads as w

    sizes = w.batch_sizes(args.instances, seed=0)
    Ss, outs = [], []
    for i, (L, N) in enumerate(sizes):
        U = w.haar_torch(L, N, seed=i)
        Ss.append(ffs.Sampler(U, flags, stream=stream))
        outs.append(torch.empty((64, N), dtype=torch.int32, device="cuda"))
    hs = [S.h for S in Ss]
    Bs = [64] * len(Ss)
    seeds = list(range(len(Ss)))

    def grouped():
        ffs.ffs_sample_batched(hs, Bs, seeds, outs, stream=stream)

    def sequential():
        for S, o, sd in zip(Ss, outs, seeds):
            ffs.ffs_sample_ex(S.h, 64, sd, 0, 0, o, stream=stream)

    res = {}
    for name, fn in (("grouped", grouped), ("sequential", sequential)):
        fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        res[name] = {"ms": e0.elapsed_time(e1), "wall_ms": 1e3 * (time.perf_counter() - t0)}
    total = 64 * len(Ss)
    flops = sum(flops_per_sample(L, N, True) for L, N in sizes) * 64
    for S in Ss:
        S.close()
    return {"workload": f"{len(Ss)} Haar complex instances, L log-uniform [256, 8192], N log-uniform "
                        f"[16, min(1024, L/4)], 64 samples each",
            "samples": total, "grouped_samples_per_s": total / (res["grouped"]["ms"] / 1e3),
            "sequential_samples_per_s": total / (res["sequential"]["ms"] / 1e3),
            "grouped_over_sequential": res["sequential"]["ms"] / res["grouped"]["ms"],
            "grouped_ms": res["grouped"]["ms"], "sequential_ms": res["sequential"]["ms"],
            "residual_algorithmic_tflops": flops / (res["grouped"]["ms"] / 1e3) / 1e12,
            "launch": "one CUDA graph of grouped launches"}


def bench_reweight(x, spec, stream, reps=20):
    """Slater-Jastrow reweighting of the last timed batch: nearest-neighbour density-density
    Jastrow (V = 0.05 per bond) and a random one-body observable, whole call timed
    (kernels, result copy and synchronisation)."""
    import torch

    from paper_2109_07358_gb300 import ffs
    from paper_2109_07358_gb300 import workloads as w

    B, n_occ = int(x.shape[0]), int(x.shape[1])
    nx, ny = spec["grid"]
    v = tuple(torch.from_numpy(a).cuda() for a in w.neighbour_jastrow_csr(nx, ny, 0.05))
    o = torch.from_numpy(np.random.default_rng(0).standard_normal(nx * ny)).cuda()
    torch.cuda.synchronize()
    ffs.ffs_jastrow_estimate(x, nx * ny, v, o, None, stream=stream)
    walls = []
    for _ in range(reps):
        t0 = time.perf_counter()
        r = ffs.ffs_jastrow_estimate(x, nx * ny, v, o, None, stream=stream)
        walls.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.median(walls))
    return {"jastrow": f"nearest-neighbour, V=0.05 per bond, {int(v[2].numel())} entries", "B": B,
            "n_occ": n_occ, "ms_per_call": ms, "samples_per_s": B / (ms / 1e3), "mean": r["mean"],
            "ess": r["ess"], "timing": "host wall clock of the synchronous call, median of 20"}


def bench_lensemble(flags, stream, B=4096, reps=3):
    """L-ensemble DPP sampling (text-summarisation stand-in): L = 16384 items, D = 512
    quality-scaled Gaussian features (alpha = 0.08, expected 126 kept eigenvectors), the
    rank-512 eigenbasis on the device, B samples per call; each call keeps eigenvectors,
    reads the longest chain back and runs the chains.  Host wall clock per call (the call
    synchronises once inside) and CUDA-event time, median of `reps` after one warm-up."""
    import torch

    from paper_2109_07358_gb300 import ffs
    from paper_2109_07358_gb300 import workloads as w

    L, D, alpha = 16384, 512, 0.08
    Phi = torch.from_numpy(w.lensemble_quality_features(L, D, alpha, seed=0)).cuda()
    Uf, sv, _ = torch.linalg.svd(Phi, full_matrices=False)
    lam = (sv * sv).contiguous()
    V = Uf.contiguous()
    torch.cuda.synchronize()
    S = ffs.Sampler(V, flags, stream=stream)
    S.sample_lensemble(lam, B, 0, stream=stream)
    S.sync()
    walls, evs = [], []
    for r in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        out = S.sample_lensemble(lam, B, 1 + r, stream=stream)
        e1.record(stream)
        S.sync()
        walls.append(time.perf_counter() - t0)
        evs.append(e0.elapsed_time(e1))
    n = out["n"].double()
    S.close()
    ms = 1e3 * float(np.median(walls))
    flops = float((L * n * (n + 1)).sum())  # the paper's 2Lk per step, summed over each chain
    return {"workload": f"L-ensemble, L={L} items, D={D} features x quality (alpha={alpha}), rank-{D} "
                        f"eigenbasis, B={B}", "samples_per_s": B / (ms / 1e3), "ms_per_call": ms,
            "event_ms_per_call": float(np.median(evs)), "mean_kept": float(n.mean()),
            "max_kept": int(n.max()), "expected_kept": float((lam / (lam + 1)).sum()),
            "algorithmic_tflops": flops / (ms / 1e3) / 1e12}


def bench_grouped(U, flags, B, L, N, cplx, peaks, args, stream):
    """The opt-in grouped form on the same workload: 128 samples share a column order, so
    step k contracts only k+1 columns (the paper's 2Lk count).  One warm-up and one timed
    call; the residual phase's algorithmic rate against the mode's tensor peak."""
    import torch

    from paper_2109_07358_gb300 import ffs

    S = ffs.Sampler(U, flags | ffs.FFS_FORM_GROUPED, stream=stream)
    x = torch.empty((B, N), dtype=torch.int32, device="cuda")
    ffs.ffs_sample_ex(S.h, B, 0, 0, 0, x, stream=stream)
    S.sync()
    ffs.ffs_profile(S.h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ffs.ffs_sample_ex(S.h, B, 1, 0, 0, x, stream=stream)
    e1.record(stream)
    S.sync()
    ms = e0.elapsed_time(e1)
    prof = ffs.ffs_profile_read(S.h)
    ffs.ffs_profile(S.h, False)
    S.close()
    res_ms = prof["residual"][0]
    mult = {"bf16x3": 3, "fp32": 1, "tf32": 1, "bf16": 1}[args.chosen]
    peak = peaks["bf16_sus"] / (2 if args.chosen == "tf32" else mult)
    alg = flops_per_sample(L, N, cplx) * B / (res_ms / 1e3) / 1e12
    return {"form": "grouped column order (128 samples per group)", "samples_per_s": B / (ms / 1e3),
            "ms_per_step": ms, "residual_ms": res_ms, "residual_algorithmic_tflops": alg,
            "residual_frac_of_tensor_peak": alg / peak, "tensor_peak_tflops": peak,
            "note": "samples of a group share m (each sample is exact, the group's samples are dependent)"}


def bench_metropolis(flags, stream, B=4096, reps=3):
    """Large-L variant (Supplementary Section S-7): open chain of L = 2^20 sites, N = 128,
    m_cond = 64 Metropolis updates per step; CUDA-event time per call of B samples,
    median of `reps` after one warm-up, next to one call of the exact all-site path on
    the same handle."""
    import torch

    from paper_2109_07358_gb300 import ffs
    from paper_2109_07358_gb300 import workloads as w

    L, N, M = 1 << 20, 128, 64
    U = torch.from_numpy(w.open_chain(L, N)).cuda()
    torch.cuda.synchronize()
    S = ffs.Sampler(U, flags, stream=stream)
    x = torch.empty((B, N), dtype=torch.int32, device="cuda")

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        S.sync()
        return e0.elapsed_time(e1)

    def mcmc(seed):
        return lambda: ffs.ffs_sample_metropolis(S.h, B, seed, 0, 0, M, x, stream=stream)

    timed(mcmc(0))
    ms = float(np.median([timed(mcmc(1 + r)) for r in range(reps)]))
    ffs.ffs_sample_ex(S.h, 64, 0, 0, 0, x[:64], stream=stream)
    S.sync()
    ms_exact = timed(lambda: ffs.ffs_sample_ex(S.h, B, 0, 0, 0, x, stream=stream))
    S.close()
    return {"workload": f"open chain L={L}, N={N}, m_cond={M}, B={B}", "samples_per_s": B / (ms / 1e3),
            "ms_per_call": ms, "exact_path_ms_per_call": ms_exact,
            "exact_path_samples_per_s": B / (ms_exact / 1e3)}


def bench_serving(args, flags):
    """Poisson streams of projection-DPP requests (U = top-N left singular vectors of L
    unit-norm Gaussian features of dimension D; L log-uniform [500, 20000], D in [64, 512],
    N in [5, min(200, D)], 1-32 samples) into the continuous-batching engine.  First the
    saturated throughput (every request submitted at once), then Poisson arrivals at
    fractions of it; latency is submission to completion (p50 / p99 / mean per rate)."""
    import numpy as np

    from paper_2109_07358_gb300 import ffs
    from paper_2109_07358_gb300 import workloads as w

    sizes = w.serving_requests(args.requests, seed=0)
    Us = [w.lensemble_orbitals_torch(L, D, N, seed=1000 + i).cpu().numpy() for i, (L, D, N, _) in enumerate(sizes)]
    outs = [np.empty((s, N), dtype=np.int32) for (L, D, N, s) in sizes]
    samples = sum(s for (_, _, _, s) in sizes)

    def run(rate):
        gaps = np.random.default_rng(1).exponential(1.0 / rate, size=len(sizes)) if rate else np.zeros(len(sizes))
        srv = ffs.ffs_server_create(0, flags, 0)
        ids = []
        t0 = time.perf_counter()
        t_next = t0
        for i, (L, D, N, s) in enumerate(sizes):
            t_next += gaps[i]
            while time.perf_counter() < t_next:
                time.sleep(0.0002)
            ids.append(ffs.ffs_submit(srv, Us[i], ffs.FFS_F64, L, N, s, 7 + i, outs[i]))
        lat = [ffs.ffs_wait(srv, rid, 600_000) for rid in ids]
        wall = time.perf_counter() - t0
        st = ffs.ffs_server_stats(srv)
        ffs.ffs_server_destroy(srv)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(np.mean(lat)), "samples_per_s": samples / wall,
                "requests_per_s": len(sizes) / wall, "engine_iterations": st["iterations"],
                "peak_requests_per_iteration": st["peak_active"]}

    run(0)  # warm-up: tile tuning of the size classes, allocator
    sat = run(0)
    sat_rps = sat["requests_per_s"]
    sweep = []
    for f in args.serving_fractions:
        r = run(f * sat_rps)
        r["fraction_of_saturated"] = f
        r["offered_requests_per_s"] = f * sat_rps
        sweep.append(r)
    return {"workload": f"{len(sizes)} L-ensemble requests, L log-uniform [500, 20000], D uniform [64, 512], "
                        f"N uniform [5, min(200, D)], 1-32 samples ({samples} samples)",
            "saturated": sat, "sweep": sweep,
            "latency": "submission to completion per request (ffs_wait), p50 / p99 over the requests"}


def bench_latency_chain(flags, stream, calls=200):
    """Per-call latency of the small plain workload (open chain L = 64, N = 8, B = 10^4,
    seed 0): each call has its own CUDA events; its working set fits in L2, so a 516 MB
    buffer is written between calls, outside the events."""
    import torch

    from paper_2109_07358_gb300 import ffs
    from paper_2109_07358_gb300 import workloads as w

    U = torch.from_numpy(w.chain_L64_N8()).cuda()
    B = 10_000
    S = ffs.Sampler(U, flags, stream=stream)
    x = torch.empty((B, 8), dtype=torch.int32, device="cuda")
    flush = torch.empty(4 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    for i in range(3):
        ffs.ffs_sample_ex(S.h, B, 0, 0, 0, x, stream=stream)
    S.sync()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
    with torch.cuda.stream(stream):
        for i in range(calls):
            flush.fill_(i)
            evs[i][0].record(stream)
            ffs.ffs_sample_ex(S.h, B, 0, 0, 0, x, stream=stream)
            evs[i][1].record(stream)
    S.sync()
    ms = np.array([a.elapsed_time(b) for a, b in evs])
    S.close()
    return {"workload": "chain64_N8_B10000", "calls": calls, "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)), "samples_per_s": B / (float(np.median(ms)) / 1e3),
            "l2": "516 MB written between calls, outside the events"}


# ------------------------------------------------------------------------------ GPU path
def run_timed(S, B, steps, warmup, rank, world, stream, x, local, flush_needed, n_steps=0):
    """W warm-up calls, then K timed calls of B samples (each with its own CUDA events on
    the handle's stream, per-phase profiling on, clocks sampled meanwhile)."""
    import torch

    from paper_2109_07358_gb300 import ffs
    from paper_2109_07358_gb300.shard import step_offset

    def step(i):
        ffs.ffs_sample_ex(S.h, B, 0, step_offset(i, rank, world, B), n_steps, x, stream=stream)

    for i in range(warmup):
        step(i)
    S.sync()
    flush = torch.empty(4 * L2_BYTES // 4, dtype=torch.int32, device="cuda") if flush_needed else None
    ffs.ffs_profile(S.h, True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    return step, flush, evs


def kernel_launches(res_n, tail_n, panel_n, pans_n, ptc_n, perm_n, N, nb=32):
    """Kernel launches behind the profiler's phase counts.  Each phase count is one timed
    region; with the tensor-core trailing update a panel end's regions hold several
    kernels: the new rows are C's slices + ozy_kernel (ozy alone when no old rows exist,
    k0 = 0), the old rows are two slice kernels + the product + the next operand (the
    operand alone at k0 = 0)."""
    n = res_n + tail_n + panel_n + pans_n + ptc_n + perm_n
    if ptc_n:
        ends = sum(1 for k0 in range(0, N, nb) if min(k0 + nb, N) < N)  # panel ends per wave-step
        first = panel_n / ends if ends else 0                          # those with k0 = 0
        n += (panel_n - first) + 3 * (ptc_n - first)
    return int(round(n))


def phase_report(prof, L, N, B, K, cplx, chosen, state, peaks, trailing_tc):
    """Per-phase times and rates, the residual (GEMM) roofline against the tensor-core
    peak of its precision, and the state update's dominant kernel against its peak."""
    res_ms, res_n = prof["residual"]
    tail_ms, tail_n = prof["tail"]
    panel_ms, panel_n = prof["panel"]
    pans_ms, pans_n = prof["panel_s"]
    ptc_ms, ptc_n = prof["panel_tc"]
    perm_ms, perm_n = prof["perm"]
    res_flops = flops_per_sample(L, N, cplx) * B * K
    issued = (2 * (2 * L) * (2 * N) * N if cplx else 2 * L * N * N) * B * K
    bf = {k: v * B * K for k, v in blocked_flops_per_sample(N, cplx).items()}
    mult = {"bf16x3": 3, "fp32": 1, "tf32": 1, "bf16": 1}[chosen]

    def tfl(fl, ms):
        return fl / (ms / 1e3) / 1e12 if ms else None

    if chosen == "fp32":
        res_peak, res_bound, res_src = NOMINAL_FP32_TFLOPS, "alu", "nominal FP32 rate (CUDA cores)"
        tensor_peak = None
    else:
        tensor_peak = peaks["bf16_sus"] / (2 if chosen == "tf32" else 1)
        res_peak, res_bound = tensor_peak / mult, "tensor"
        res_src = (f"{peaks['source']} bf16_tflops_sustained {peaks['bf16_sus']}" +
                   {"bf16x3": " / 3 (three BF16 products per term)", "tf32": " / 2 (TF32 rate)", "bf16": ""}[chosen])
    ach = tfl(res_flops, res_ms)
    roof = {"kernel": "residual_tc_kernel" if chosen != "fp32" else "residual_fp32_kernel", "phase": "residual (GEMM)",
            "bound": res_bound, "achieved": ach, "peak": res_peak, "unit": "TFLOP/s",
            "frac": ach / res_peak if ach else None,
            "issued_achieved": tfl(issued * mult, res_ms) if tensor_peak else None,
            "issued_frac": (tfl(issued * mult, res_ms) / tensor_peak) if tensor_peak and res_ms else None,
            "traffic": None, "peak_source": res_src + " (measured; the kernel runs inside a long step)",
            "algorithmic": "the paper's 2Lk flops per sample-step, L N (N+1) per sample" + (" x4 complex" if cplx else ""),
            "per_launch": "algorithmic flops of all residual launches / their summed CUDA-event time"}
    e = {"df64": 8, "fp64": 8, "fp32": 4}[state] * (2 if cplx else 1)
    gsum = 0 if chosen == "fp32" else (16 if cplx else 32)  # the tensor-core residual writes group sums
    bb = {k: v * B * K for k, v in blocked_bytes_per_sample(L, N, e, gsum=gsum).items()}

    def gbs(by, ms):
        return by / (ms / 1e3) / 1e9 if ms else None

    # with the tensor-core trailing update both halves of the panel end run on tcgen05:
    # the new rows (FFS_PHASE_PANEL: C's slices + ozy_kernel) and Top (FFS_PHASE_PANEL_TC)
    new_tc = bool(ptc_n) and trailing_tc
    phases = {
        "residual": {"kernel": roof["kernel"], "ms": res_ms / K, "launches_per_step": res_n / K,
                     "algorithmic_tflops": ach, "issued_tflops": tfl(issued * mult, res_ms)},
        "tail_step": {"kernel": "tail_step_kernel", "ms": tail_ms / K, "launches_per_step": tail_n / K,
                      "algorithmic_tflops": tfl(bf["step"], tail_ms), "algorithmic_gbs": gbs(bb["step"], tail_ms)},
        "tail_panel_s": {"kernel": "tail_panel_s_kernel", "ms": pans_ms / K, "launches_per_step": pans_n / K,
                         "algorithmic_tflops": tfl(bf["panel_s"], pans_ms)},
        "tail_panel": {"kernel": "ozy_kernel (+ C slices)" if new_tc else "tail_panel_kernel",
                       "ms": panel_ms / K, "launches_per_step": panel_n / K,
                       "algorithmic_tflops": tfl(bf["panel"] - (bf["top"] if ptc_n else 0.0), panel_ms),
                       **({"algorithmic_gbs": gbs(bb["new"], panel_ms)} if new_tc else {})},
        "perm": {"kernel": "perm_init_kernel", "ms": perm_ms / K, "launches_per_step": perm_n / K},
    }
    if ptc_n:
        phases["tail_panel_tc"] = {"kernel": "oz_top_kernel (+ slices, operand)", "ms": ptc_ms / K,
                                   "launches_per_step": ptc_n / K, "algorithmic_tflops": tfl(bf["top"], ptc_ms),
                                   "algorithmic_gbs": gbs(bb["top"], ptc_ms)}
    total_ms = max(1e-9, res_ms + tail_ms + panel_ms + pans_ms + ptc_ms + perm_ms)
    # the state update's dominant phase: a memory-bound one (the per-step update, or the
    # tensor-core panel-end halves, whose issued BF16 products per state byte sit below the
    # tensor ridge) against the measured HBM copy rate; the CUDA-core new-row kernel
    # against the derived peak of its own arithmetic
    cands = {"tail_step": tail_ms, "tail_panel": panel_ms}
    if ptc_n:
        cands["tail_panel_tc"] = ptc_ms
    dom = max(cands, key=cands.get)
    if dom != "tail_panel" or new_tc:
        by = {"tail_step": bb["step"], "tail_panel": bb["new"], "tail_panel_tc": bb["top"]}[dom]
        a_gbs = gbs(by, cands[dom])
        roof_tail = {"kernel": phases[dom]["kernel"], "phase": dom, "bound": "hbm", "achieved": a_gbs,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": a_gbs / peaks["hbm_gbs"] if a_gbs else None, "traffic": None,
                     "peak_source": f"{peaks['source']} hbm_gbs (copy bandwidth)",
                     "algorithmic": {"tail_step": "per sample-step: the weights' group sums and the chosen group (or "
                                                  "all L weights), the live panel block read and written back, W0_P "
                                                  "at a panel's first step",
                                     "tail_panel": "per sample-panel: W0_T read, the new rows' U entries read and the new "
                                                   "rows written",
                                     "tail_panel_tc": "per sample-panel: W0_T read and Top written, W0_P read"}[dom]
                                    + f" ({e}-byte entries)",
                     "share_of_step": cands[dom] / total_ms}
        launches = kernel_launches(res_n, tail_n, panel_n, pans_n, ptc_n, perm_n, N) // K
        return phases, roof, roof_tail, launches
    # the CUDA-core new-row kernel against the peak of its own arithmetic
    if state == "df64":
        instr = DF_INSTR_COMPLEX if cplx else DF_INSTR_REAL
        st_peak = FP32_INSTR_PER_S / instr * (8 if cplx else 2) / 1e12
        st_src = (f"derived: {FP32_INSTR_PER_S / 1e12:.1f} T FP32 instructions/s (152 SMs x 128 lanes x 2.07 GHz) / "
                  f"{instr} instructions per {'complex (Karatsuba)' if cplx else 'real'} double-float multiply-add "
                  f"x {8 if cplx else 2} flops")
    elif state == "fp64":
        st_peak, st_src = NOMINAL_FP64_TFLOPS, "nominal FP64 rate (1.25 TFLOP/s; 1.22 measured by an FMA loop)"
    else:
        st_peak, st_src = NOMINAL_FP32_TFLOPS, "nominal FP32 rate (152 SMs x 128 lanes x 2 x 2.07 GHz)"
    fl_panel = bf["panel"] - (bf["top"] if ptc_n else 0.0)
    tail_ach = tfl(fl_panel, panel_ms)
    roof_tail = {"kernel": f"tail_panel_kernel ({state} state)", "phase": "tail_panel", "bound": "alu",
                 "achieved": tail_ach, "peak": st_peak, "unit": "TFLOP/s",
                 "frac": tail_ach / st_peak if tail_ach else None,
                 "traffic": None, "peak_source": st_src, "share_of_step": panel_ms / total_ms}
    launches = kernel_launches(res_n, tail_n, panel_n, pans_n, ptc_n, perm_n, N) // K
    return phases, roof, roof_tail, launches

def section(out, name, fn):
    """Run an optional section; a failure is recorded in the line instead of losing it."""
    t0 = time.perf_counter()
    try:
        out[name] = fn()
    except Exception as e:  # noqa: BLE001 - the headline must survive a failing extra section
        out[name] = {"error": f"{type(e).__name__}: {e}"}
    if isinstance(out[name], dict):
        out[name]["section_wall_s"] = round(time.perf_counter() - t0, 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ffs", choices=["ffs", "reference"])
    ap.add_argument("--workload", default="anderson_L16384_N2048_B8192", choices=list(WORKLOADS))
    ap.add_argument("--B", type=int, default=0, help="override samples per step")
    ap.add_argument("--chosen", default="bf16x3", choices=["bf16x3", "fp32", "tf32", "bf16"])
    ap.add_argument("--state", default="df64", choices=["df64", "fp64", "fp32"])
    ap.add_argument("--no-trailing-tc", dest="trailing_tc", action="store_false",
                    help="keep the once-per-panel trailing update on the CUDA cores (default: tensor cores)")
    ap.add_argument("--plain-B", type=int, default=512, help="samples of the timed plain-form call")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-samples", type=int, default=0)
    ap.add_argument("--no-lattice", action="store_true", help="skip the 64x64 lattice section")
    ap.add_argument("--no-fp64-state", action="store_true", help="skip the IEEE FP64 state section")
    ap.add_argument("--no-latency", action="store_true", help="skip the per-call latency of the L = 64 chain")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-marginal", action="store_true")
    ap.add_argument("--marginal-steps", type=int, default=128)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-reweight", action="store_true")
    ap.add_argument("--no-lensemble", action="store_true")
    ap.add_argument("--no-metropolis", action="store_true")
    ap.add_argument("--no-grouped", action="store_true")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--serving-fractions", type=float, nargs="*", default=[0.25, 0.5, 0.75, 0.9, 1.1])
    args = ap.parse_args()
    spec = dict(WORKLOADS[args.workload])
    if args.B:
        spec["B"] = args.B

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, spec, rank, world)

    import torch

    from paper_2109_07358_gb300 import build as _build
    from paper_2109_07358_gb300 import ffs

    _build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    peaks = load_peaks()
    U_np = make_U(spec)
    L, N = U_np.shape
    cplx = np.iscomplexobj(U_np)
    B = spec["B"]
    U = torch.from_numpy(U_np).cuda()
    res_flag = {"bf16x3": ffs.FFS_RES_BF16X3, "fp32": ffs.FFS_RES_FP32, "tf32": ffs.FFS_RES_TF32,
                "bf16": ffs.FFS_RES_BF16}[args.chosen]
    state_flag = {"df64": ffs.FFS_STATE_DF64, "fp64": ffs.FFS_STATE_FP64, "fp32": ffs.FFS_STATE_FP32}[args.state]

    def flags_for(is_cplx):
        # the trailing update on the tensor cores (double-float state, tensor-core residual)
        tc = args.trailing_tc and args.state == "df64" and args.chosen != "fp32"
        return res_flag | state_flag | (ffs.FFS_TRAILING_TC if tc else 0)

    flags = flags_for(cplx)
    flags_real = flags_for(False)  # the sections with real or mixed U
    stream = torch.cuda.Stream()
    S = ffs.Sampler(U, flags, stream=stream)
    x = torch.empty((B, N), dtype=torch.int32, device="cuda")
    # a working set that fits in L2 twice over is evicted between timed steps by writing a
    # buffer larger than L2, outside the per-step events; otherwise the steps run back to
    # back and each step's inputs are larger than L2 already
    ws = working_set_bytes(L, N, B, cplx, args.state)
    step, flush, evs = run_timed(S, B, args.steps, args.warmup, rank, world, stream, x, local, ws < 2 * L2_BYTES)
    barrier()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")   # lets a profiler capture the timed steps only
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                if flush is not None:
                    flush.fill_(i)
                evs[i][0].record(stream)
                step(args.warmup + i)
                evs[i][1].record(stream)
        S.sync()
        torch.cuda.nvtx.range_pop()
    barrier()
    step_ms = np.array([a.elapsed_time(b) for a, b in evs])
    ms_total = float(step_ms.sum())
    prof = ffs.ffs_profile_read(S.h)
    ffs.ffs_profile(S.h, False)
    del flush
    if dist is not None:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    value = world * B / (ms_step / 1e3)
    phases, roof, roof_tail, launches = phase_report(prof, L, N, B, args.steps, cplx, args.chosen, args.state, peaks,
                                                     bool(flags & ffs.FFS_TRAILING_TC))
    out = {
        "metric": "FFS samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.chosen == "fp32" else args.chosen[:4],
        "dtype_detail": {"bf16x3": "residual on tensor cores in BF16 (hi/lo split, three products, FP32 "
                                   "accumulation)", "bf16": "residual in BF16 (FP32 accumulation)",
                         "tf32": "residual in TF32 (FP32 accumulation)", "fp32": "residual in FP32 on CUDA cores"}
        [args.chosen] + f"; {args.state} state" + (" (pairs of FP32 numbers)" if args.state == "df64" else ""),
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": spec["desc"], "L": L, "N": N, "B": B,
                   "form": f"batched {args.chosen} residual + {args.state} state" +
                           (" + tensor-core trailing update" if flags & ffs.FFS_TRAILING_TC else ""),
                   "working_set_bytes": ws,
                   "l2": "inputs larger than L2 (steps back to back)" if ws >= 2 * L2_BYTES else
                   "working set below L2: a 516 MB buffer is written between timed steps, outside their "
                   "CUDA events"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "calls": int(args.steps), "what": "one ffs_sample_ex call of B samples (CUDA events)"},
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_tail": roof_tail,
        "phases": phases,
    }
    main_sections(args, out, ffs, torch, S, U, U_np, spec, flags, flags_real, stream, x, B, L, N, cplx, peaks,
                  ms_step, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main_sections(args, out, ffs, torch, S, U, U_np, spec, flags, flags_real, stream, x, B, L, N, cplx, peaks,
                  ms_step, rank, world):
    """The sections after the headline (rank 0 only, except the end-to-end line)."""
    from paper_2109_07358_gb300.shard import step_offset

    def timed_call(h, n, seed, xo, n_steps=0):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ffs.ffs_sample_ex(h, n, seed, 0, n_steps, xo, stream=stream)
        e1.record(stream)
        ffs.ffs_sync(h)
        return e0.elapsed_time(e1)

    if not args.no_plain and rank == 0:
        def plain():
            nb = min(B, args.plain_B)
            P = ffs.Sampler(U, ffs.FFS_FORM_PLAIN, stream=stream)
            xp = torch.empty((nb, N), dtype=torch.int32, device="cuda")
            ffs.ffs_sample_ex(P.h, min(nb, 64), 0, 0, 0, xp, stream=stream)
            P.sync()
            pms = timed_call(P.h, nb, 0, xp)
            P.close()
            return {"value": nb / (pms / 1e3), "unit": "samples/s", "ms_per_call": pms, "B": nb,
                    "form": "plain per-sample FP32 (CUDA cores, FP32 state)",
                    "chosen_over_plain": out["value"] / world / (nb / (pms / 1e3)),
                    "note": f"samples 0..{nb - 1} of the same workload (the plain form's rate does not grow with B "
                            "once the GPU is full)"}
        section(out, "plain", plain)

    if not args.no_cpu and rank == 0:
        def cpu():
            n, threads = oracle_plan(U_np, B)
            rate, wall, workers = oracle_baseline(U_np, n, threads=threads)
            return {"value": rate, "unit": "samples/s", "cores": workers, "kind": "oracle",
                    "sample": f"{n} samples of the same workload (indices 0..{n - 1}), {wall:.1f} s wall, "
                              + ("one single-threaded worker per core" if threads == 1 else
                                 f"one process, BLAS on {workers} threads")}
        section(out, "cpu_baseline", cpu)

    if not args.no_marginal and rank == 0:
        def marginal():
            nm = min(args.marginal_steps, N)
            xm = torch.empty((B, nm), dtype=torch.int32, device="cuda")
            ffs.ffs_sample_ex(S.h, B, 0, 0, nm, xm, stream=stream)
            S.sync()
            mms = timed_call(S.h, B, 0, xm, nm)
            return {"n_steps": nm, "samples_per_s": B / (mms / 1e3), "ms_per_batch": mms,
                    "full_chain_ms_per_batch": ms_step}
        section(out, "marginal", marginal)
    if not args.no_reweight and rank == 0:
        section(out, "reweight", lambda: bench_reweight(x, spec, stream))
    S.close()
    if not args.no_e2e:
        def e2e():
            # End to end through the C ABI with host buffers: U uploaded from pinned host
            # memory (ffs_create_ex), samples read back into pinned host memory.  Runs after
            # the device-timed handle is released, so that both see the same free memory.
            U_host = torch.from_numpy(U_np).pin_memory()
            x_host = torch.empty((B, N), dtype=torch.int32).pin_memory()
            times = []
            for i in range(args.e2e_steps + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = ffs.ffs_create_ex(U_host, ffs.dtype_of(U_host), L, N, N, flags, stream)
                ffs.ffs_sample_ex(h, B, 0, step_offset(i, rank, world, B), 0, x_host, stream=stream)
                ffs.ffs_destroy(h)
                times.append(time.perf_counter() - t0)
            e2e_s = float(np.median(times[1:]))
            return {"value": world * B / e2e_s, "unit": "samples/s",
                    "h2d_bytes_per_step": int(U_host.numel() * U_host.element_size()),
                    "d2h_bytes_per_step": int(x_host.numel() * 4), "steps": args.e2e_steps,
                    "what": "host wall clock of ffs_create_ex (U from pinned host memory) + ffs_sample_ex into "
                            "pinned host memory + ffs_destroy, median of the timed steps after one warm-up"}
        section(out, "e2e", e2e)
    if rank != 0:
        return
    if not args.no_latency:
        section(out, "latency_chain64", lambda: bench_latency_chain(flags_for_chain(ffs, args), stream))
    if not args.no_lattice and args.workload != "lattice64x64_N1024_B4096":
        section(out, "lattice", lambda: bench_lattice(args, ffs, torch, stream, peaks))
    if not args.no_fp64_state:
        section(out, "fp64_state", lambda: bench_fp64_state(args, ffs, torch, stream))
    if not args.no_lensemble:
        section(out, "lensemble", lambda: bench_lensemble(flags_real, stream))
    if not args.no_grouped:
        section(out, "grouped", lambda: bench_grouped_lattice(args, ffs, torch, stream, peaks))
    if not args.no_metropolis:
        section(out, "metropolis", lambda: bench_metropolis(flags_real, stream))
    if not args.no_batching:
        section(out, "batching", lambda: bench_batching(args, res_and_state(ffs, args) |
                                                        (ffs.FFS_TRAILING_TC if args.trailing_tc and
                                                         args.state == "df64" and args.chosen != "fp32" else 0),
                                                        stream))
    if not args.no_serving:
        section(out, "serving", lambda: bench_serving(args, flags_real))


def res_and_state(ffs, args):
    return ({"bf16x3": ffs.FFS_RES_BF16X3, "fp32": ffs.FFS_RES_FP32, "tf32": ffs.FFS_RES_TF32,
             "bf16": ffs.FFS_RES_BF16}[args.chosen] |
            {"df64": ffs.FFS_STATE_DF64, "fp64": ffs.FFS_STATE_FP64, "fp32": ffs.FFS_STATE_FP32}[args.state])


def flags_for_chain(ffs, args):
    return res_and_state(ffs, args)


def lattice_flags(ffs, args, state=None):
    st = state or args.state
    tc = args.trailing_tc and st == "df64" and args.chosen != "fp32"
    return ({"bf16x3": ffs.FFS_RES_BF16X3, "fp32": ffs.FFS_RES_FP32, "tf32": ffs.FFS_RES_TF32,
             "bf16": ffs.FFS_RES_BF16}[args.chosen] |
            {"df64": ffs.FFS_STATE_DF64, "fp64": ffs.FFS_STATE_FP64, "fp32": ffs.FFS_STATE_FP32}[st] |
            (ffs.FFS_TRAILING_TC if tc else 0))


_LATTICE = {}


def lattice_U(torch):
    if "U" not in _LATTICE:
        from paper_2109_07358_gb300 import workloads as w

        _LATTICE["np"] = w.lattice_64x64_N1024(0)
        _LATTICE["U"] = torch.from_numpy(_LATTICE["np"]).cuda()
    return _LATTICE["U"]


def bench_lattice(args, ffs, torch, stream, peaks, steps=3):
    """The 64 x 64 random-phase lattice (L = 4096, N = 1024, complex, B = 4096) in the
    chosen form: one warm-up and `steps` timed calls with per-phase profiling."""
    U = lattice_U(torch)
    L, N, B = 4096, 1024, 4096
    S = ffs.Sampler(U, lattice_flags(ffs, args), stream=stream)
    x = torch.empty((B, N), dtype=torch.int32, device="cuda")
    ffs.ffs_sample_ex(S.h, B, 0, 0, 0, x, stream=stream)
    S.sync()
    ffs.ffs_profile(S.h, True)
    ms = []
    for i in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ffs.ffs_sample_ex(S.h, B, 0, (1 + i) * B, 0, x, stream=stream)
        e1.record(stream)
        S.sync()
        ms.append(e0.elapsed_time(e1))
    prof = ffs.ffs_profile_read(S.h)
    S.close()
    phases, roof, roof_tail, launches = phase_report(prof, L, N, B, steps, True, args.chosen, args.state, peaks,
                                                     args.trailing_tc)
    m = float(np.mean(ms))
    return {"workload": "lattice64x64_N1024_B4096", "samples_per_s": B / (m / 1e3), "ms_per_step": m,
            "steps": steps, "roofline": roof, "roofline_tail": roof_tail, "phases": phases}


def bench_fp64_state(args, ffs, torch, stream):
    """The IEEE FP64 state against the chosen double-float state on the 64 x 64 lattice
    (B = 4096, one timed call each after a 128-sample warm-up): the price of IEEE FP64 on
    GB300's FP64 pipes."""
    U = lattice_U(torch)
    B, N = 4096, 1024
    x = torch.empty((B, N), dtype=torch.int32, device="cuda")
    res = {}
    for st in ("fp64", "df64"):
        S = ffs.Sampler(U, lattice_flags(ffs, args, st), stream=stream)
        ffs.ffs_sample_ex(S.h, 128, 0, 0, 0, x[:128], stream=stream)
        S.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ffs.ffs_sample_ex(S.h, B, 0, 0, 0, x, stream=stream)
        e1.record(stream)
        S.sync()
        S.close()
        ms = e0.elapsed_time(e1)
        res[st] = {"samples_per_s": B / (ms / 1e3), "ms_per_call": ms}
    res["workload"] = "lattice64x64_N1024_B4096"
    res["df64_over_fp64"] = res["df64"]["samples_per_s"] / res["fp64"]["samples_per_s"]
    return res


def bench_grouped_lattice(args, ffs, torch, stream, peaks):
    """The opt-in grouped form on the 64 x 64 lattice (one call after a warm-up)."""
    U = lattice_U(torch)
    return bench_grouped(U, lattice_flags(ffs, args), 4096, 4096, 1024, True, peaks, args, stream)


if __name__ == "__main__":
    sys.exit(main())
