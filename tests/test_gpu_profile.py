"""Per-phase profiling (ffs_profile / ffs_profile_read) on the GPU: the launches it
counts are the ones the blocked schedule makes, its times are positive, enabling clears
the totals, and profiling does not change the samples."""
import numpy as np
import pytest
import torch

from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_07358_gb300.build import build

    build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("N,n_steps", [(75, 0), (75, 40), (64, 0)])
def test_phase_launch_counts(N, n_steps):
    U = torch.from_numpy(w.haar(200, N, seed=3)).cuda()
    S = ffs.Sampler(U, ffs.FFS_RES_BF16X3 | ffs.FFS_STATE_DF64)
    ref = S.sample(70, 5, n_steps=n_steps)["x"].clone()
    S.sync()
    ffs.ffs_profile(S.h, True)
    got = S.sample(70, 5, n_steps=n_steps)["x"]
    prof = ffs.ffs_profile_read(S.h)
    S.sync()
    assert torch.equal(ref, got)
    K = n_steps or N
    panels_with_trailing = len([k1 for k1 in range(32, K, 32)])   # panel ends that have columns left
    assert prof["perm"][1] == 1
    assert prof["residual"][1] == K
    assert prof["tail"][1] == K
    assert prof["panel_s"][1] == panels_with_trailing
    assert prof["panel"][1] == panels_with_trailing
    for name, (ms, n) in prof.items():
        if n:
            assert ms > 0.0, name
    ffs.ffs_profile(S.h, True)          # enabling again clears the totals
    assert all(n == 0 for _, n in ffs.ffs_profile_read(S.h).values())
    ffs.ffs_profile(S.h, False)
    S.close()


def test_metropolis_phases_and_marginal_chain():
    from oracle import ffs_oracle as orc

    U = w.haar(300, 70, seed=4, complex_=False)
    S = ffs.Sampler(torch.from_numpy(U).cuda(), ffs.FFS_STATE_DF64)
    ffs.ffs_profile(S.h, True)
    X = S.sample_metropolis(24, 16, 7, n_steps=45)["x"].cpu().numpy()
    prof = ffs.ffs_profile_read(S.h)
    S.sync()
    S.close()
    assert prof["residual"][1] == 0 and prof["tail"][1] == 45 and prof["panel"][1] == 1
    same = 0
    for s in range(24):
        r = orc.sample_one_metropolis(U, 16, 7, s, n_steps=45, record=True)
        d = np.nonzero(X[s] != r["x"])[0]
        if d.size == 0:
            same += 1
        else:
            assert r["margin"][d[0]] <= 1e-9
    assert same >= 22
