"""The two multi-instance patterns against standalone sampling.

Batching: many instances of uneven L and N in one grouped, graph-captured schedule
must give, for every instance, exactly the samples of a standalone ffs_sample call.
Serving: requests submitted at different times (continuous batching, admission by
device-memory budget) must each give exactly their standalone samples, whatever else
shares the GPU with them.
"""
import time

import numpy as np
import pytest
import torch

from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w

pytestmark = pytest.mark.gpu

FLAGS = ffs.FFS_RES_BF16X3 | ffs.FFS_STATE_DF64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_07358_gb300.build import build

    build()
    assert torch.cuda.is_available()


def standalone(U, B, seed, flags=FLAGS):
    S = ffs.Sampler(torch.from_numpy(U).cuda(), flags)
    x = S.sample(B, seed)["x"].cpu().numpy()
    S.sync()
    S.close()
    return x


@pytest.mark.parametrize("cplx", [True, False])
def test_batched_instances_equal_standalone(cplx):
    sizes = [(300, 40, 70), (1000, 100, 130), (256, 16, 64), (700, 75, 1), (128, 33, 200)]
    Us = [w.haar(L, N, seed=10 + i, complex_=cplx) for i, (L, N, _) in enumerate(sizes)]
    Ss = [ffs.Sampler(torch.from_numpy(U).cuda(), FLAGS) for U in Us]
    outs = [torch.full((B, U.shape[1]), -1, dtype=torch.int32, device="cuda") for U, (_, _, B) in zip(Us, sizes)]
    seeds = [100 + i for i in range(len(sizes))]
    for rep in range(2):  # twice: the second call reuses the workspaces
        ffs.ffs_sample_batched([S.h for S in Ss], [B for (_, _, B) in sizes], seeds, outs)
        for S in Ss:
            S.sync()
        for i, (U, (L, N, B)) in enumerate(zip(Us, sizes)):
            assert np.array_equal(outs[i].cpu().numpy(), standalone(U, B, seeds[i])), (rep, i)
    for S in Ss:
        S.close()


def test_batched_rejects_mixed_configurations():
    a = ffs.Sampler(torch.from_numpy(w.haar(64, 8, seed=1)).cuda(), FLAGS)
    b = ffs.Sampler(torch.from_numpy(w.haar(64, 8, seed=2, complex_=False)).cuda(), FLAGS)
    outs = [torch.empty((4, 8), dtype=torch.int32, device="cuda") for _ in range(2)]
    with pytest.raises(ffs.FFSError) as e:
        ffs.ffs_sample_batched([a.h, b.h], [4, 4], [0, 0], outs)
    assert e.value.code == ffs.FFS_E_ARG


def _requests(n, seed=0):
    r = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        L = int(r.integers(200, 1500))
        D = int(r.integers(16, 64))
        N = int(r.integers(5, min(60, D)))
        ns = int(r.integers(1, 33))
        U = w.lensemble_orbitals(w.lensemble_features(L, D, seed=1000 + i), N)
        reqs.append((U, ns, 7 + i))
    return reqs


def test_server_requests_equal_standalone_in_a_mix():
    reqs = _requests(12)
    srv = ffs.ffs_server_create(0, FLAGS, 6)
    outs = [np.full((ns, U.shape[1]), -1, dtype=np.int32) for U, ns, _ in reqs]
    ids = [None] * len(reqs)
    lat = [None] * len(reqs)
    try:
        # half up front, the rest arriving while the first ones are on the GPU
        for i in range(6):
            U, ns, sd = reqs[i]
            ids[i] = ffs.ffs_submit(srv, U, ffs.dtype_of(U), U.shape[0], U.shape[1], ns, sd, outs[i])
        time.sleep(0.005)
        for i in range(6, 12):
            U, ns, sd = reqs[i]
            ids[i] = ffs.ffs_submit(srv, U, ffs.dtype_of(U), U.shape[0], U.shape[1], ns, sd, outs[i])
        for i in range(12):
            lat[i] = ffs.ffs_wait(srv, ids[i], 60_000)
        stats = ffs.ffs_server_stats(srv)
    finally:
        ffs.ffs_server_destroy(srv)
    for i, (U, ns, sd) in enumerate(reqs):
        assert np.array_equal(outs[i], standalone(U, ns, sd)), i
    assert stats["active"] == 0 and stats["pending"] == 0
    print("latencies ms:", [round(x, 2) for x in lat], "iterations", stats["iterations"])


def test_server_admission_budget_and_rejection():
    reqs = _requests(4, seed=1)
    U0 = reqs[0][0]
    # a budget that fits roughly one request at a time: the rest queue, all complete
    srv = ffs.ffs_server_create(64 << 20, FLAGS, 0)
    try:
        outs = [np.full((ns, U.shape[1]), -1, dtype=np.int32) for U, ns, _ in reqs]
        ids = [ffs.ffs_submit(srv, U, ffs.dtype_of(U), U.shape[0], U.shape[1], ns, sd, o)
               for (U, ns, sd), o in zip(reqs, outs)]
        for i in ids:
            ffs.ffs_wait(srv, i, 60_000)
        for (U, ns, sd), o in zip(reqs, outs):
            assert np.array_equal(o, standalone(U, ns, sd))
        big = w.haar(20000, 500, seed=3, complex_=False)
        with pytest.raises(ffs.FFSError) as e:
            ffs.ffs_submit(srv, big, ffs.FFS_F64, 20000, 500, 32, 0, np.empty((32, 500), np.int32))
        assert e.value.code == ffs.FFS_E_NOMEM
    finally:
        ffs.ffs_server_destroy(srv)
