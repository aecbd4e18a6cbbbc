"""The grouped form (FFS_FORM_GROUPED): the 128 samples of a group share the column order
of the group's first sample index, and each step contracts only the leading columns of
that order.  Checked against the oracle run with the same orders:

* column orders bit-exact and shared within each group; teacher-forced conditionals
  within the chosen form's 1e-4 (real, complex, three panels; ragged last group,
  first_sample_index a nonzero multiple of 128); free-running draws identical up to
  excused CDF boundaries; a sample does not depend on the batch it is drawn in;
* the set distribution over many groups against brute force |det U_S|^2 (chi-squared);
* argument errors and the calls that do not take the form.
"""
from collections import Counter

import numpy as np
import pytest
import torch
from scipy.stats import chisquare

from oracle import ffs_oracle as orc
from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w
from tests.parity_util import cdf_error, draw_identity, window

pytestmark = pytest.mark.gpu

G = ffs.FFS_FORM_GROUPED
SEED = 4242
CASES = {
    "real": lambda: w.haar(300, 40, seed=1, complex_=False),
    "complex": lambda: w.haar(200, 30, seed=2),
    "panels": lambda: w.haar(160, 75, seed=9),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_07358_gb300.build import build

    build()
    assert torch.cuda.is_available()


def sampler(U, flags):
    return ffs.Sampler(torch.from_numpy(np.ascontiguousarray(U)).cuda(), flags)


def oracle_grouped(U, samples):
    N = U.shape[1]
    return [orc.sample_one(U, SEED, s, m=orc.permutation(SEED, s // 128 * 128, N), record=True) for s in samples]


_R = {}


@pytest.mark.parametrize("state", ["df64", "fp64"])
@pytest.mark.parametrize("case", list(CASES))
def test_parity(case, state):
    U = CASES[case]()
    B, first = 300, 128
    if case not in _R:
        _R[case] = oracle_grouped(U, range(first, first + B))
    recs = _R[case]
    flags = G | ffs.FFS_RES_BF16X3 | (ffs.FFS_STATE_DF64 if state == "df64" else ffs.FFS_STATE_FP64)
    S = sampler(U, flags)
    out = S.sample(B, SEED, first_sample_index=first, perm=True)
    S.sync()
    X, P = out["x"].cpu().numpy(), out["perm"].cpu().numpy()
    for b, r in enumerate(recs):
        assert np.array_equal(P[b], r["m"])
    g = (np.arange(B) + first) // 128
    for gi in np.unique(g):
        rows = P[g == gi]
        assert (rows == rows[0]).all()
    force = torch.tensor(np.stack([r["x"] for r in recs]), dtype=torch.int32, device="cuda")
    outf = S.sample(B, SEED, first_sample_index=first, force_x=force, probs=True)
    S.sync()
    Pf = outf["probs"].cpu().double().numpy()
    err = float(np.abs(Pf - np.stack([r["probs"] for r in recs])).max())
    meas = cdf_error(Pf, recs)
    eps = window(meas, False)
    frac, bad = draw_identity(X, recs, eps=eps)
    print(f"grouped {case} {state}: measured CDF error {meas:.2e}, eps {eps:.2e}, unexcused {bad}")
    assert not bad
    # a sample is the same when drawn in a smaller batch
    part = S.sample(128, SEED, first_sample_index=first + 128)["x"].cpu().numpy()
    S.sync()
    S.close()
    assert np.array_equal(part, X[128:256])
    print(f"grouped {case} {state}: max |dP| = {err:.2e}, identical samples {frac:.3f}")
    assert err <= 1e-4


def test_distribution_over_many_groups():
    U = w.haar(8, 3, seed=6, complex_=False)
    P = orc.set_probabilities(U)
    B = 128 * 300
    S = sampler(U, G | ffs.FFS_RES_BF16X3 | ffs.FFS_STATE_DF64)
    X = S.sample(B, 11)["x"].cpu().numpy()
    S.sync()
    S.close()
    cnt = Counter(tuple(sorted(r.tolist())) for r in X)
    keys = list(P)
    obs = np.array([cnt.get(k, 0) for k in keys], dtype=float)
    exp = np.array([P[k] * B for k in keys])
    assert obs.sum() == B
    p = chisquare(obs, exp * obs.sum() / exp.sum()).pvalue
    print(f"grouped form, 300 groups: chi-squared p = {p:.3f}")
    assert p > 1e-3


def test_errors():
    U = w.haar(64, 8, seed=3, complex_=False)
    Ud = torch.from_numpy(U).cuda()
    with pytest.raises(ffs.FFSError) as e:
        ffs.Sampler(Ud, G | ffs.FFS_RES_FP32)
    assert e.value.code == ffs.FFS_E_ARG
    with pytest.raises(ffs.FFSError) as e:
        ffs.Sampler(Ud, G | ffs.FFS_TAIL_UNBLOCKED)
    assert e.value.code == ffs.FFS_E_ARG
    S = ffs.Sampler(Ud, G | ffs.FFS_RES_BF16X3 | ffs.FFS_STATE_DF64)
    with pytest.raises(ffs.FFSError) as e:
        S.sample(4, 0, first_sample_index=5)
    assert e.value.code == ffs.FFS_E_ARG
    with pytest.raises(ffs.FFSError) as e:
        S.sample_lensemble(np.ones(8), 4, 0)
    assert e.value.code == ffs.FFS_E_UNSUPPORTED
    with pytest.raises(ffs.FFSError) as e:
        S.sample_metropolis(4, 8)
    assert e.value.code == ffs.FFS_E_UNSUPPORTED
    x = torch.empty((4, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(ffs.FFSError):
        ffs.ffs_sample_batched([S.h], [4], [0], [x])
    S.close()
