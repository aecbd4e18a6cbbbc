"""Helpers shared by the GPU parity tests: oracle runs and the draw-identity rule."""
import numpy as np

from oracle import ffs_oracle as o


def oracle_runs(U, seed, samples, n_steps=None):
    """Oracle records (x, m, probs, u, logp) for the given sample indices."""
    return [o.sample_one(U, seed, s, n_steps=n_steps, record=True) for s in samples]


def _runs_worker(args):
    U, seed, lo, hi, n_steps = args
    return [o.sample_one(U, seed, s, n_steps=n_steps, record=True) for s in range(lo, hi)]


def oracle_runs_parallel(U, seed, lo, hi, n_steps=None, workers=None):
    """Oracle records for samples lo..hi-1 over a spawn-started pool (safe after CUDA init)."""
    import multiprocessing as mp
    import os

    workers = max(1, min(workers or os.cpu_count() or 1, hi - lo))
    bounds = np.linspace(lo, hi, workers + 1).astype(int)
    jobs = [(U, seed, int(bounds[i]), int(bounds[i + 1]), n_steps) for i in range(workers)]
    with mp.get_context("spawn").Pool(workers, initializer=o._single_thread) as pool:
        parts = pool.map(_runs_worker, jobs)
    return [r for p in parts for r in p]


def first_divergence(xg, xo):
    d = np.nonzero(np.asarray(xg) != np.asarray(xo))[0]
    return int(d[0]) if d.size else -1


def excused(rec, k, xg, eps):
    """A differing draw at step k is excused when the uniform lies within eps of an
    oracle CDF boundary between the oracle's site and the GPU's site (both sides then
    place the same step on opposite sides of a boundary that rounding can move)."""
    P = rec["probs"][k]
    F = np.cumsum(P)
    u = rec["u"][k]
    xo = int(rec["x"][k])
    lo, hi = min(xo, int(xg)), max(xo, int(xg))
    bounds = F[lo:hi]
    return bool(bounds.size) and float(np.min(np.abs(bounds - u))) <= eps


def draw_identity(X_gpu, recs, eps):
    """(fraction of identical samples, list of unexcused divergences)."""
    same = 0
    bad = []
    for b, rec in enumerate(recs):
        k = first_divergence(X_gpu[b], rec["x"])
        if k < 0:
            same += 1
        elif not excused(rec, k, X_gpu[b][k], eps):
            bad.append((b, k, int(X_gpu[b][k]), int(rec["x"][k])))
    return same / max(1, len(recs)), bad
