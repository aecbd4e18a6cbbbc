"""Slater-Jastrow reweighting on the GPU (Supplementary Section S-5) against the oracle.

* Element-wise parity of the per-sample log J^2 and o_L, and of the four results, on
  random configurations with random sparse and dense v, o, q; ragged batch sizes, a
  full lattice (n_occ = n_orb) and an orbital count that needs the large shared-memory
  bitmap.
* Invalid configurations and matrices are reported as FFS_E_ARG.
* The Anderson-Hubbard workload of the main text (4 x 4 lattice, 4 + 4 fermions,
  Gutzwiller factor of Eq. 4): 10^6 GPU samples per spin species, reweighted on the GPU,
  against the exact enumeration of all 1820^2 configurations, within 5 standard errors.
* The 64 x 64 lattice batch (4096 samples of 1024 fermions) with a nearest-neighbour
  Jastrow: per-sample parity on sampled rows and the results against the oracle.
"""
import itertools

import numpy as np
import pytest
import torch

from oracle import ffs_oracle as orc
from paper_2109_07358_gb300 import ffs
from paper_2109_07358_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_07358_gb300.build import build

    build()
    assert torch.cuda.is_available()


def dense(csr, n):
    rowptr, col, val = csr
    m = np.zeros((n, n))
    for i in range(n):
        np.add.at(m[i], col[rowptr[i]:rowptr[i + 1]], val[rowptr[i]:rowptr[i + 1]])
    return m


def random_csr(rng, n, density):
    m = (rng.random((n, n)) < density) * rng.standard_normal((n, n))
    rowptr = np.zeros(n + 1, np.int64)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(m[i])[0]
        rowptr[i + 1] = rowptr[i] + nz.size
        cols.append(nz)
        vals.append(m[i, nz])
    return rowptr, np.concatenate(cols).astype(np.int32), np.concatenate(vals)


def to_dev(csr):
    if csr is None:
        return None
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in csr)


def run(X, n_orb, v=None, o=None, q=None):
    xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.int32)).cuda()
    B = X.shape[0]
    lj = torch.empty(B, dtype=torch.float64, device="cuda")
    ob = torch.empty(B, dtype=torch.float64, device="cuda")
    od = None if o is None else torch.from_numpy(o).cuda()
    r = ffs.ffs_jastrow_estimate(xd, n_orb, to_dev(v), od, to_dev(q), lj, ob)
    return r, lj.cpu().numpy(), ob.cpu().numpy()


def restrict(X, csr, keep):
    """The rows and columns ``keep`` of a CSR matrix, dense (n^T v n only involves
    occupied orbitals, so the oracle can work on the orbitals that the samples use)."""
    if csr is None:
        return None
    pos = {int(k): i for i, k in enumerate(keep)}
    rowptr, col, val = csr
    m = np.zeros((len(keep), len(keep)))
    for k in keep:
        for e in range(rowptr[k], rowptr[k + 1]):
            if int(col[e]) in pos:
                m[pos[int(k)], pos[int(col[e])]] += val[e]
    return m


def compare(X, n_orb, v, o, q):
    r, lj, ob = run(X, n_orb, v, o, q)
    keep = np.unique(X)
    Xr = np.searchsorted(keep, X)
    vr = restrict(X, v, keep)
    ref = orc.jastrow_reweight(Xr, np.zeros((keep.size, keep.size)) if vr is None else vr,
                               o=None if o is None else o[keep], q=restrict(X, q, keep))
    scale = 1.0 + np.abs(ref["logj2"]).max()
    assert np.abs(lj - ref["logj2"]).max() <= 1e-13 * scale
    assert np.abs(ob - ref["obs"]).max() <= 1e-13 * (1.0 + np.abs(ref["obs"]).max())
    for k in ("mean", "log_j2_mean", "ess", "stderr"):
        assert r[k] == pytest.approx(ref[k], rel=1e-10, abs=1e-13), k
    return r


@pytest.mark.parametrize("n_orb,n_occ,B,density", [(40, 7, 1, 0.3), (40, 7, 13, 0.3), (97, 31, 1001, 0.1),
                                                   (64, 64, 9, 0.5), (256, 100, 300, 1.0),
                                                   (70000, 12, 37, 0.0)])
def test_parity_random(n_orb, n_occ, B, density):
    rng = np.random.default_rng(n_orb * 1000 + B)
    X = np.stack([rng.permutation(n_orb)[:n_occ] for _ in range(B)])
    if density > 0:
        v, q = random_csr(rng, n_orb, density), random_csr(rng, n_orb, density)
    else:  # large orbital count: Gutzwiller-like, one entry per row
        half = n_orb // 2
        v = w.gutzwiller_csr(half, 1.3)
        q = w.gutzwiller_csr(half, 2.0)
    o = rng.standard_normal(n_orb)
    compare(X, n_orb, v, o, q)
    compare(X, n_orb, None, o, None)
    compare(X, n_orb, v, None, None)


def test_deterministic():
    rng = np.random.default_rng(7)
    X = np.stack([rng.permutation(300)[:50] for _ in range(5000)])
    v = random_csr(rng, 300, 0.2)
    o = rng.standard_normal(300)
    a, b = run(X, 300, v, o), run(X, 300, v, o)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])


@pytest.mark.parametrize("case", ["repeat", "range", "negative", "col", "rowptr"])
def test_invalid_inputs(case):
    n = 16
    X = np.array([[0, 1, 2], [3, 4, 5]])
    v = w.gutzwiller_csr(n // 2, 1.0)
    if case == "repeat":
        X[1, 2] = 3
    elif case == "range":
        X[0, 1] = n
    elif case == "negative":
        X[1, 0] = -1
    elif case == "col":
        v = (v[0], v[1].copy(), v[2])
        v[1][4] = n + 5
    elif case == "rowptr":
        v = (v[0].copy(), v[1], v[2])
        v[0][5] = v[0][-1] + 3   # rows 4 and 5 (occupied in the second sample) run past nnz
    with pytest.raises(ffs.FFSError) as e:
        run(X, n, v)
    assert e.value.code == ffs.FFS_E_ARG


def test_anderson_hubbard_4x4_against_exact_enumeration():
    L, V = 16, 2.0
    U = w.anderson_hubbard_4x4(W=2.0, seed=0)
    sets = list(itertools.combinations(range(L), 4))
    p = np.array([np.linalg.det(U[list(S), :]) ** 2 for S in sets])
    mask = np.array([sum(1 << i for i in S) for S in sets], dtype=np.int64)
    both = mask[:, None] & mask[None, :]
    d = np.zeros(both.shape)
    for i in range(L):
        d += (both >> i) & 1
    n0 = ((mask[:, None] & 1) + (mask[None, :] & 1)).astype(float)
    P = np.outer(p, p) * np.exp(-V * d)
    D_ex, n0_ex = (P * d).sum() / P.sum(), (P * n0).sum() / P.sum()

    B = 1_000_000
    S = ffs.Sampler(torch.from_numpy(U).cuda(), ffs.FFS_RES_FP32 | ffs.FFS_STATE_FP64)
    xu = S.sample(B, 1)["x"]
    xd = S.sample(B, 2)["x"]
    S.sync()
    S.close()
    X = torch.cat([xu, xd + L], dim=1).contiguous()
    g = to_dev(w.gutzwiller_csr(L, V))
    o = torch.zeros(2 * L, dtype=torch.float64, device="cuda")
    o[0] = o[L] = 1.0
    q = to_dev((np.arange(2 * L + 1).clip(max=L).astype(np.int64), np.arange(L, 2 * L).astype(np.int32),
                np.ones(L)))
    rn = ffs.ffs_jastrow_estimate(X, 2 * L, g, o, None)
    rD = ffs.ffs_jastrow_estimate(X, 2 * L, g, None, q)
    print(f"4x4 Anderson-Hubbard V={V}: <n_0> {rn['mean']:.5f} +- {rn['stderr']:.5f} (exact {n0_ex:.5f}), "
          f"<D> {rD['mean']:.5f} +- {rD['stderr']:.5f} (exact {D_ex:.5f}), ESS {rn['ess']:.0f} of {B}")
    assert abs(rn["mean"] - n0_ex) < 5 * rn["stderr"]
    assert abs(rD["mean"] - D_ex) < 5 * rD["stderr"]


def test_lattice_batch_neighbour_jastrow():
    U = w.lattice_64x64_N1024(0)
    S = ffs.Sampler(torch.from_numpy(U).cuda(), ffs.FFS_RES_BF16X3 | ffs.FFS_STATE_DF64)
    X = S.sample(4096, 0)["x"]
    S.sync()
    S.close()
    v = w.neighbour_jastrow_csr(64, 64, 0.05)
    rng = np.random.default_rng(1)
    o = rng.standard_normal(4096)
    lj = torch.empty(4096, dtype=torch.float64, device="cuda")
    ob = torch.empty(4096, dtype=torch.float64, device="cuda")
    r = ffs.ffs_jastrow_estimate(X, 4096, to_dev(v), torch.from_numpy(o).cuda(), None, lj, ob)
    Xh = X.cpu().numpy()
    ref = orc.jastrow_reweight(Xh, dense(v, 4096), o=o)
    assert np.abs(lj.cpu().numpy() - ref["logj2"]).max() <= 1e-12
    assert np.abs(ob.cpu().numpy() - ref["obs"]).max() <= 1e-11
    for k in ("mean", "log_j2_mean", "ess", "stderr"):
        assert r[k] == pytest.approx(ref[k], rel=1e-10), k
