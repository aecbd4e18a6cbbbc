"""Large-L Metropolis draws on the GPU (ffs_sample_metropolis, Supplementary Section
S-7) against the oracle.

* Same random numbers, same chains: the GPU's samples equal the oracle's except where a
  chain decision came within the state precision of flipping (the oracle records each
  step's closest decision; a divergence is excused only at a step whose margin is below
  the mode's bound).  Column orders bit-exact.  Real, complex and multi-panel cases.
* A 2^20-site open chain with N = 128 (the regime the variant is for): sampled outputs
  against the oracle one by one.
* The chain's output distribution: site occupations of 2 x 10^4 samples on a 4096-site
  chain against the exact one-body density sum_n |U_yn|^2.
* Argument errors.
"""
import numpy as np
import pytest
import torch

from oracle import ffs_oracle as orc
from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w

pytestmark = pytest.mark.gpu

SEED = 99
MODES = {
    "fp64": (ffs.FFS_STATE_FP64, 1e-9),
    "df64": (ffs.FFS_STATE_DF64, 1e-9),
    "fp32": (ffs.FFS_STATE_FP32, 1e-4),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_07358_gb300.build import build

    build()
    assert torch.cuda.is_available()


def sampler(U, flags):
    return ffs.Sampler(torch.from_numpy(np.ascontiguousarray(U)).cuda(), flags)


def check_against_oracle(U, X, perm, samples, m_cond, margin_bound, n_steps=None):
    same = 0
    for i, s in enumerate(samples):
        r = orc.sample_one_metropolis(U, m_cond, SEED, s, n_steps=n_steps, record=True)
        if perm is not None:
            assert np.array_equal(perm[i], r["m"])
        d = np.nonzero(X[i] != r["x"])[0]
        if d.size == 0:
            same += 1
        else:
            k = int(d[0])
            assert r["margin"][k] <= margin_bound, (s, k, r["margin"][k])
    return same


_CASES = {
    "real": lambda: w.haar(300, 40, seed=1, complex_=False),
    "complex": lambda: w.haar(200, 30, seed=2),
    "panels": lambda: w.haar(160, 75, seed=9),
}


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("case", list(_CASES))
def test_parity(case, mode):
    flags, bound = MODES[mode]
    U = _CASES[case]()
    B, M = 40, 24
    S = sampler(U, flags)
    out = S.sample_metropolis(B, M, SEED, perm=True)
    S.sync()
    S.close()
    X, P = out["x"].cpu().numpy(), out["perm"].cpu().numpy()
    same = check_against_oracle(U, X, P, range(B), M, bound)
    print(f"Metropolis {case} {mode}: identical samples {same}/{B}")
    assert same >= 0.9 * B


def test_large_L_chain():
    L, N, M, B = 1 << 20, 128, 64, 4096
    U = w.open_chain(L, N)
    S = sampler(U, ffs.FFS_STATE_DF64)
    X = S.sample_metropolis(B, M, SEED)["x"].cpu().numpy()
    S.sync()
    S.close()
    assert all(len(set(row.tolist())) == N for row in X[:256])   # no site twice
    picks = [0, 1, 2, 2049, 4095]
    same = check_against_oracle(U, X[picks], None, picks, M, 1e-9)
    print(f"Metropolis L=2^20 N=128 m_cond=64: identical sampled outputs {same}/{len(picks)}")
    assert same >= len(picks) - 1


def test_occupations_match_the_one_body_density():
    L, N, M, B = 4096, 64, 200, 20000
    U = w.open_chain(L, N)
    S = sampler(U, ffs.FFS_STATE_DF64)
    X = S.sample_metropolis(B, M, 5)["x"]
    S.sync()
    S.close()
    occ = torch.bincount(X.flatten().long(), minlength=L).cpu().numpy() / B
    rho = orc.one_body_density(U)
    z = (occ - rho) / np.sqrt(rho * (1 - rho) / B)
    print(f"Metropolis occupations: max |z| over {L} sites = {np.abs(z).max():.2f}")
    assert np.abs(z).max() < 5.5
    assert abs(occ.sum() - N) < 1e-9


def test_argument_errors():
    U = w.haar(64, 8, seed=3, complex_=False)
    S = sampler(U, ffs.FFS_STATE_DF64)
    x = torch.empty((4, 8), dtype=torch.int32, device="cuda")
    for args in ((4, 0, 0, 0, -1), (4, 0, 0, 9, 10), (4, 0, 0, 8, 1 << 30)):
        with pytest.raises(ffs.FFSError) as e:
            ffs.ffs_sample_metropolis(S.h, *args, x)
        assert e.value.code == ffs.FFS_E_ARG
    with pytest.raises(ffs.FFSError) as e:
        ffs.ffs_sample_metropolis(S.h, 4, 0, 0, 0, 10, np.zeros((4, 8), np.int32))
    assert e.value.code == ffs.FFS_E_ARG
    S.close()
    S = sampler(U, ffs.FFS_FORM_PLAIN)
    with pytest.raises(ffs.FFSError) as e:
        S.sample_metropolis(4, 10)
    assert e.value.code == ffs.FFS_E_UNSUPPORTED
    S.close()
