"""Parity at the full sizes of the configured workloads, on outputs the oracle can
compute one sample at a time.

* 64 x 64 random-phase lattice (L = 4096, N = 1024, complex), B = 4096 in the launch
  configuration the benchmark times (BF16x3 residual, double-float state, the old rows'
  trailing update on the tensor cores): no site twice in any of the 4096 samples, and
  free-running draws of sampled indices against the oracle (identical except within
  the tolerance window of a CDF boundary); teacher-forced conditionals of four samples
  for the chosen residual form (1e-4) and the FP32 path (1e-6).
* Anderson chain (L = 16384, N = 2048, real): teacher-forced conditionals of two
  samples, per residual precision, against the FP64 oracle; the error table is printed.
  Free running at the benchmark's size and form (B = 8192, two waves of the 34 MB
  per-sample state): no site twice in any sample, and four sampled indices spread over
  both waves identical to the oracle's free-running samples except at boundary cases
  within the excusal window.
Excusal windows are the CDF errors measured teacher-forced on the same samples (floor
1e-6; tests/parity_util.py).
"""
import numpy as np
import pytest
import torch

from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w
from tests.parity_util import (cdf_error, draw_identity, forced_draw_identity, forced_probs, oracle_runs_at,
                               oracle_runs_parallel, window)

pytestmark = pytest.mark.gpu

CHOSEN = ffs.FFS_RES_BF16X3 | ffs.FFS_STATE_DF64
BENCH_FORM = CHOSEN | ffs.FFS_TRAILING_TC  # what bench.py times


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_07358_gb300.build import build

    build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def lattice():
    U = w.lattice_64x64_N1024(0)
    recs = oracle_runs_parallel(U, 0, 0, 16)
    return U, recs


def test_lattice_full_batch_draws(lattice):
    U, recs = lattice
    S = ffs.Sampler(torch.from_numpy(U).cuda(), BENCH_FORM)
    X = S.sample(4096, 0)["x"].cpu().numpy()
    S.sync()
    S.close()
    assert ((X >= 0) & (X < U.shape[0])).all()
    assert (np.diff(np.sort(X, axis=1), axis=1) > 0).all()  # no site twice in any sample
    S = ffs.Sampler(torch.from_numpy(U).cuda(), BENCH_FORM)
    P = forced_probs(S, recs, 0)
    S.close()
    meas = cdf_error(P, recs)
    eps = window(meas, False)
    frac, bad = draw_identity(X[:16], recs, eps=eps)
    fd, nd = forced_draw_identity(P, recs)
    # a whole sample is 1024 chained draws: one boundary case anywhere changes the rest
    print(f"lattice 64x64 full batch: {frac:.3f} of sampled whole samples identical, teacher-forced draws "
          f"{fd:.5f} of {nd}, measured CDF error {meas:.2e}, eps {eps:.2e}, unexcused {bad}")
    assert not bad
    assert fd >= 0.999


@pytest.mark.parametrize("flags,tol", [(CHOSEN, 1e-4), (ffs.FFS_RES_FP32 | ffs.FFS_STATE_DF64, 1e-6)])
def test_lattice_teacher_forced(lattice, flags, tol):
    U, recs = lattice
    S = ffs.Sampler(torch.from_numpy(U).cuda(), flags)
    force = torch.tensor(np.stack([r["x"] for r in recs[:4]]), dtype=torch.int32, device="cuda")
    out = S.sample(4, 0, force_x=force, probs=True)
    S.sync()
    err = 0.0
    draws = same = 0
    for b in range(4):
        P = out["probs"][b].cpu().double().numpy()
        err = max(err, float(np.abs(P - recs[b]["probs"]).max()))
        # per-draw identity: the site the GPU conditional gives for the shared uniform
        C = np.cumsum(P, axis=1)
        for k in range(P.shape[0]):
            u = recs[b]["u"][k]
            hit = np.nonzero((C[k] > u * C[k, -1]) & (P[k] > 0))[0]
            xg = int(hit[0]) if hit.size else int(np.nonzero(P[k] > 0)[0][-1])
            draws += 1
            same += xg == int(recs[b]["x"][k])
    S.close()
    print(f"lattice 64x64 teacher-forced flags={flags:#x}: max |dP| = {err:.3e}, identical draws {same}/{draws}")
    assert err <= tol
    assert same >= 0.999 * draws


def test_anderson_precision_table():
    U = w.anderson_L16384_N2048(0)
    recs = oracle_runs_parallel(U, 0, 0, 2)
    force = torch.tensor(np.stack([r["x"] for r in recs]), dtype=torch.int32, device="cuda")
    table = {}
    modes = {"bf16x3": (ffs.FFS_RES_BF16X3, 1e-4), "bf16x3_tc": (ffs.FFS_RES_BF16X3 | ffs.FFS_TRAILING_TC, 1e-4),
             "tf32": (ffs.FFS_RES_TF32, None), "bf16": (ffs.FFS_RES_BF16, None), "fp32": (ffs.FFS_RES_FP32, 1e-6)}
    Ud = torch.from_numpy(U).cuda()
    for name, (res, tol) in modes.items():
        S = ffs.Sampler(Ud, res | ffs.FFS_STATE_DF64)
        out = S.sample(2, 0, force_x=force, probs=True)
        S.sync()
        err = max(float(np.abs(out["probs"][b].cpu().double().numpy() - recs[b]["probs"]).max()) for b in range(2))
        S.close()
        table[name] = err
        if tol is not None:
            assert err <= tol, (name, err)
    print("Anderson L=16384 N=2048 max |dP| vs FP64 oracle:", {k: f"{v:.2e}" for k, v in table.items()})


def test_anderson_full_batch_free_running():
    """B = 8192 in the benchmark's form; indices 0, 1 (first wave) and 4097, 8191 (second
    wave, when the batch runs in two) against the oracle's free-running samples."""
    U = w.anderson_L16384_N2048(0)
    idx = [0, 1, 4097, 8191]
    recs = oracle_runs_at(U, 0, idx)
    S = ffs.Sampler(torch.from_numpy(U).cuda(), BENCH_FORM)
    X = S.sample(8192, 0)["x"].cpu().numpy()
    S.sync()
    assert ((X >= 0) & (X < U.shape[0])).all()
    assert (np.diff(np.sort(X, axis=1), axis=1) > 0).all()  # no site twice in any sample
    P = [forced_probs(S, [r], 0, first=s)[0] for s, r in zip(idx, recs)]
    S.close()
    meas = cdf_error(P, recs)
    eps = window(meas, False)
    frac, bad = draw_identity(X[idx], recs, eps=eps)
    fd, nd = forced_draw_identity(P, recs)
    print(f"Anderson full batch: {frac:.3f} of sampled whole samples identical, teacher-forced draws {fd:.5f} "
          f"of {nd}, measured CDF error {meas:.2e}, eps {eps:.2e}, unexcused {bad}")
    assert not bad
    assert fd >= 0.999
