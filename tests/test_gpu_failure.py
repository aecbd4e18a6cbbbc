"""Failure paths, exercised without faulting, trapping or hanging the GPU.

* A bounded wait that runs out: ffs_debug_inject arms a one-shot fault for the next
  tensor-core residual launch (the TMA producer of its first CTA skips one pipeline
  stage and the launch's waits give up after 4096 polls).  ffs_sync must report
  FFS_E_TIMEOUT, and the same handle must then sample exactly as a fresh handle does.
* A vanishing normaliser: U with a zero column (created with FFS_NO_ORTHO_CHECK) makes
  every weight of the step whose column it is zero, so the chain reports FFS_E_NUMERIC
  at ffs_sync, on the tensor-core, FP32 and plain forms; the context stays usable.
"""
import numpy as np
import pytest
import torch

from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w

pytestmark = pytest.mark.gpu

CHOSEN = ffs.FFS_RES_BF16X3 | ffs.FFS_STATE_DF64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_07358_gb300.build import build

    build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("cplx", [False, True])
def test_wait_that_runs_out_reports_timeout_and_the_handle_recovers(cplx):
    U = torch.from_numpy(w.haar(300, 40, seed=21, complex_=cplx)).cuda()
    S = ffs.Sampler(U, CHOSEN)
    ref = S.sample(70, 5)["x"].clone()
    S.sync()
    ffs.ffs_debug_inject(S.h, ffs.FFS_FAULT_SKIP_ARRIVAL)
    S.sample(70, 5)
    with pytest.raises(ffs.FFSError) as e:
        S.sync()
    assert e.value.code == ffs.FFS_E_TIMEOUT
    again = S.sample(70, 5)["x"]
    S.sync()  # the status word was cleared and the call succeeded
    assert torch.equal(again, ref)
    fresh = ffs.Sampler(U, CHOSEN)
    assert torch.equal(fresh.sample(70, 5)["x"], ref)
    fresh.sync()
    fresh.close()
    S.close()


def test_inject_argument_checks():
    U = torch.from_numpy(w.haar(64, 8, seed=2)).cuda()
    S = ffs.Sampler(U, ffs.FFS_RES_FP32)
    with pytest.raises(ffs.FFSError) as e:
        ffs.ffs_debug_inject(S.h, ffs.FFS_FAULT_SKIP_ARRIVAL)
    assert e.value.code == ffs.FFS_E_UNSUPPORTED
    with pytest.raises(ffs.FFSError) as e:
        ffs.ffs_debug_inject(S.h, 77)
    assert e.value.code == ffs.FFS_E_ARG
    ffs.ffs_debug_inject(S.h, ffs.FFS_FAULT_NONE)
    S.close()


@pytest.mark.parametrize("flags", [CHOSEN, CHOSEN | ffs.FFS_TRAILING_TC, ffs.FFS_RES_FP32 | ffs.FFS_STATE_FP64,
                                   ffs.FFS_FORM_PLAIN],
                         ids=["chosen", "trailing_tc", "fp32", "plain"])
def test_zero_column_reports_numeric(flags):
    Un = w.haar(300, 70, seed=22)
    Un[:, 17] = 0.0
    U = torch.from_numpy(np.ascontiguousarray(Un)).cuda()
    S = ffs.Sampler(U, flags | ffs.FFS_NO_ORTHO_CHECK)
    X = S.sample(40, 3)["x"]
    with pytest.raises(ffs.FFSError) as e:
        S.sync()
    assert e.value.code == ffs.FFS_E_NUMERIC
    assert int(X.min()) >= 0 and int(X.max()) < 300  # every site written stays in range
    S.close()
    good = ffs.Sampler(torch.from_numpy(w.haar(300, 70, seed=22)).cuda(), flags)
    Y = good.sample(40, 3)["x"].cpu().numpy()
    good.sync()
    good.close()
    assert (np.diff(np.sort(Y, axis=1), axis=1) > 0).all()
