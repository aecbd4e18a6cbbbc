"""Helpers shared by the GPU parity tests: oracle runs and the draw-identity rule.

Excusal window.  Given shared uniforms, a GPU draw may differ from the oracle's only
where the uniform lies within eps of an oracle CDF boundary between the two sites.
eps is 1e-6 for the FP32 path (FP32 residual, plain form, allocation-free entry
point).  For the tensor-core residual modes it is the CDF error measured on the same
samples, teacher-forced on the oracle's prefixes (the largest |F_gpu - F_oracle| over
steps and sites), with 1e-6 as the floor.  Teacher forcing reproduces the free-running
conditional of every step up to the first divergence bit for bit (a sample's arithmetic
depends only on its prefix), so a divergence needs a uniform within the measured error
of an oracle boundary.  The tests print eps next to the identity fractions.
"""
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


def _at_worker(args):
    U, seed, s, n_steps = args
    o._single_thread()
    return o.sample_one(U, seed, s, n_steps=n_steps, record=True)


def oracle_runs_at(U, seed, indices, n_steps=None):
    """Oracle records for arbitrary sample indices, one spawn-started worker each."""
    return oracle_jobs([(U, seed, int(s)) for s in indices], n_steps)


def oracle_jobs(jobs, n_steps=None):
    """Oracle records of (U, seed, sample index) jobs, possibly of different U, over a
    spawn-started pool (safe after CUDA initialisation)."""
    import multiprocessing as mp
    import os

    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_at_worker, [(U, seed, int(s), n_steps) for U, seed, s in jobs])


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


EPS_FP32 = 1e-6


def cdf_error(P_gpu, recs):
    """Largest |F_gpu - F_oracle| over samples, steps and sites, F the running sum of the
    normalised conditional in site order (P_gpu: samples x steps x L, teacher-forced)."""
    err = 0.0
    for b, rec in enumerate(recs):
        Fg = np.cumsum(np.asarray(P_gpu[b], dtype=np.float64), axis=-1)
        Fo = np.cumsum(rec["probs"], axis=-1)
        err = max(err, float(np.abs(Fg - Fo).max()))
    return err


def window(measured, fp32_path):
    """The excusal window: 1e-6 on the FP32 path, else the measured CDF error (floor 1e-6)."""
    return EPS_FP32 if fp32_path else max(EPS_FP32, float(measured))


def forced_probs(S, recs, seed, first=0):
    """Teacher-forced conditionals of the samples first .. first + len(recs) - 1 (the
    oracle's sites forced), as float64 (samples x steps x L)."""
    import torch

    force = torch.tensor(np.stack([r["x"] for r in recs]), dtype=torch.int32, device="cuda")
    out = S.sample(len(recs), seed, first_sample_index=first, force_x=force, probs=True)
    S.sync()
    return out["probs"].cpu().double().numpy()


def forced_draw_identity(P_gpu, recs):
    """Per-draw identity under teacher forcing: the fraction of steps at which the GPU's
    conditional, inverted at the shared uniform, gives the oracle's site."""
    draws = same = 0
    for b, rec in enumerate(recs):
        P = np.asarray(P_gpu[b], dtype=np.float64)
        C = np.cumsum(P, axis=1)
        for k in range(P.shape[0]):
            u = rec["u"][k]
            hit = np.nonzero((C[k] > u * C[k, -1]) & (P[k] > 0))[0]
            xg = int(hit[0]) if hit.size else int(np.nonzero(P[k] > 0)[0][-1])
            draws += 1
            same += xg == int(rec["x"][k])
    return same / max(1, draws), draws
