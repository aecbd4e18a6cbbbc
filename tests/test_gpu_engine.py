"""The two multi-instance patterns against standalone sampling.

Batching: many instances of uneven L and N in one grouped, graph-captured schedule
must give, for every instance, exactly the samples of a standalone ffs_sample call.
Serving: requests submitted at different times (continuous batching, admission by
device-memory budget) must each give exactly their standalone samples, whatever else
shares the GPU with them, and requests must actually share engine iterations.
At the configured sizes (256 Haar instances of L log-uniform in [256, 8192]; L-ensemble
requests of L up to 20000) sampled instances and requests are also compared with the
CPU oracle: free-running samples identical except at boundary cases within the excusal
window (the CDF error measured teacher-forced on the same samples, floor 1e-6).
"""
import time

import numpy as np
import pytest
import torch

from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w
from tests.parity_util import cdf_error, draw_identity, forced_probs, oracle_jobs, window

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
    print("latencies ms:", [round(x, 2) for x in lat], "iterations", stats["iterations"],
          "peak requests per iteration", stats["peak_active"])
    assert stats["peak_active"] >= 2  # requests shared engine iterations (and so their launches)


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


def _check_against_oracle(label, S, x, rec, seed, index):
    """One sample x of handle S (sample index `index`) against the oracle's record."""
    P = forced_probs(S, [rec], seed, first=index)
    meas = cdf_error(P, [rec])
    eps = window(meas, False)
    err = float(np.abs(P[0] - rec["probs"]).max())
    frac, bad = draw_identity(x[None, :], [rec], eps=eps)
    print(f"{label}: identical {frac:.0f}, max |dP| {err:.2e}, measured CDF error {meas:.2e}, eps {eps:.2e}")
    assert not bad, (label, bad)
    assert err <= 1e-4, (label, err)


def test_batching_configured_sizes_against_oracle():
    """All 256 Haar instances of the batching workload (L log-uniform in [256, 8192], N
    log-uniform in [16, min(1024, L/4)], complex, 64 samples each) in one batched call;
    the largest-L, largest-N and smallest instances and one more, against the oracle."""
    sizes = w.batch_sizes(256, seed=0)
    Us = [w.haar_torch(L, N, seed=i) for i, (L, N) in enumerate(sizes)]
    Ss = [ffs.Sampler(U, FLAGS) for U in Us]
    outs = [torch.full((64, N), -1, dtype=torch.int32, device="cuda") for (L, N) in sizes]
    seeds = list(range(len(sizes)))
    ffs.ffs_sample_batched([S.h for S in Ss], [64] * len(Ss), seeds, outs)
    for S in Ss:
        S.sync()
    for (L, N), o in zip(sizes, outs):   # every sample of every instance: N distinct sites
        X = o.cpu().numpy()
        assert ((X >= 0) & (X < L)).all() and (np.diff(np.sort(X, axis=1), axis=1) > 0).all()
    iL = int(np.argmax([L for L, _ in sizes]))
    iN = int(np.argmax([N for _, N in sizes]))
    i0 = int(np.argmin([N for _, N in sizes]))
    picks = [(iL, 63), (iN, 0), (i0, 0), (i0, 63), (2, 5)]
    Unp = {i: Us[i].cpu().numpy() for i, _ in picks}
    recs = oracle_jobs([(Unp[i], seeds[i], s) for i, s in picks])
    for (i, s), rec in zip(picks, recs):
        _check_against_oracle(f"instance {i} (L={sizes[i][0]}, N={sizes[i][1]}) sample {s}", Ss[i],
                              outs[i][s].cpu().numpy(), rec, seeds[i], s)
    for S in Ss:
        S.close()


def test_serving_configured_sizes_against_oracle_and_overlap():
    """L-ensemble requests of the serving workload's sizes (the largest L and the largest
    N of its 200 requests, and two more) in one server with smaller requests arriving
    while they run: each request's first samples against the oracle, and the engine must
    have advanced several requests in one iteration (their work shares launches)."""
    sizes = w.serving_requests(200, seed=0)
    iL = int(np.argmax([L for L, _, _, _ in sizes]))
    iN = int(np.argmax([N for _, _, N, _ in sizes]))
    big = [iL, iN, 1, 2]
    reqs = []
    for i in big:
        L, D, N, ns = sizes[i]
        U = w.lensemble_orbitals(w.lensemble_features(L, D, seed=1000 + i), N)
        reqs.append((U, ns, 7 + i))
    small = _requests(6, seed=3)
    srv = ffs.ffs_server_create(0, FLAGS, 0)
    try:
        outs = [np.full((ns, U.shape[1]), -1, dtype=np.int32) for U, ns, _ in reqs + small]
        ids = []
        for (U, ns, sd), o in zip(reqs, outs):
            ids.append(ffs.ffs_submit(srv, U, ffs.dtype_of(U), U.shape[0], U.shape[1], ns, sd, o))
        time.sleep(0.01)
        for (U, ns, sd), o in zip(small, outs[len(reqs):]):
            ids.append(ffs.ffs_submit(srv, U, ffs.dtype_of(U), U.shape[0], U.shape[1], ns, sd, o))
        for i in ids:
            ffs.ffs_wait(srv, i, 600_000)
        stats = ffs.ffs_server_stats(srv)
    finally:
        ffs.ffs_server_destroy(srv)
    print("serving: peak requests advanced in one engine iteration", stats["peak_active"])
    assert stats["peak_active"] >= 2
    for (U, ns, sd), o in zip(reqs + small, outs):
        assert np.array_equal(o, standalone(U, ns, sd))
    jobs = [(U, sd, s) for U, ns, sd in reqs for s in range(min(ns, 2))]
    recs = oracle_jobs(jobs)
    for (U, sd, s), rec in zip(jobs, recs):
        S = ffs.Sampler(torch.from_numpy(U).cuda(), FLAGS)
        j = [k for k, (Ur, _, sr) in enumerate(reqs) if sr == sd][0]
        _check_against_oracle(f"request L={U.shape[0]} N={U.shape[1]} sample {s}", S, outs[j][s], rec, sd, s)
        S.close()
