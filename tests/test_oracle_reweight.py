"""Pins of the oracle's Slater-Jastrow reweighting (Supplementary Section S-5) against
things other than itself: a hand-computed two-sample example, the special cases v = 0
and diagonal v, the invariance under a constant shift of v, exact enumeration of a small
Anderson-Hubbard system with the Gutzwiller factor of Eq. 4, and the limit of an
infinite Gutzwiller penalty."""
import itertools
import math

import numpy as np
import pytest

from oracle import ffs_oracle as orc
from paper_2109_07358_gb300 import workloads as w


def dense(csr, n):
    rowptr, col, val = csr
    m = np.zeros((n, n))
    for i in range(n):
        m[i, col[rowptr[i]:rowptr[i + 1]]] += val[rowptr[i]:rowptr[i + 1]]
    return m


def test_hand_example():
    # x_1 = {0, 1} with v_01 = v_10 = ln(2)/2: J^2 = exp(-ln 2) = 1/2; x_2 = {2, 3}: J^2 = 1.
    v = np.zeros((4, 4))
    v[0, 1] = v[1, 0] = math.log(2.0) / 2
    r = orc.jastrow_reweight([[0, 1], [2, 3]], v, o=[1.0, 0, 0, 0])
    assert r["logj2"] == pytest.approx([-math.log(2.0), 0.0], abs=1e-15)
    assert r["mean"] == pytest.approx(1.0 / 3.0, rel=1e-15)       # (1/2 * 1) / (1/2 + 1)
    assert r["log_j2_mean"] == pytest.approx(math.log(0.75), rel=1e-15)
    assert r["ess"] == pytest.approx(1.8, rel=1e-15)              # 1.5^2 / 1.25
    assert r["stderr"] == pytest.approx(math.sqrt(2.0) / 4.5, rel=1e-14)


def test_no_jastrow_is_the_plain_mean():
    rng = np.random.default_rng(3)
    X = np.stack([rng.permutation(20)[:6] for _ in range(500)])
    o = rng.standard_normal(20)
    r = orc.jastrow_reweight(X, np.zeros((20, 20)), o=o)
    obs = o[X].sum(axis=1)
    assert r["mean"] == pytest.approx(obs.mean(), rel=1e-13)
    assert r["ess"] == pytest.approx(500.0, rel=1e-13)
    assert r["log_j2_mean"] == 0.0
    assert r["stderr"] == pytest.approx(obs.std() / math.sqrt(500), rel=1e-12)


def test_diagonal_jastrow_and_pair_observable():
    rng = np.random.default_rng(4)
    X = np.stack([rng.permutation(12)[:5] for _ in range(50)])
    d = rng.standard_normal(12)
    r = orc.jastrow_reweight(X, np.diag(d), q=np.diag(d))
    # n_i^2 = n_i: a diagonal v is a one-body factor, a diagonal q a one-body observable
    assert np.allclose(r["logj2"], -d[X].sum(axis=1), atol=1e-14, rtol=0)
    assert np.allclose(r["obs"], d[X].sum(axis=1), atol=1e-14, rtol=0)


def test_constant_shift_and_order_invariance():
    rng = np.random.default_rng(5)
    X = np.stack([rng.permutation(16)[:4] for _ in range(300)])
    v = rng.standard_normal((16, 16))
    o = rng.standard_normal(16)
    a = orc.jastrow_reweight(X, v, o=o)
    b = orc.jastrow_reweight(X, v + 0.7, o=o)   # every sample has 4 particles: log J^2 - 0.7 * 16
    assert b["mean"] == pytest.approx(a["mean"], rel=1e-12)
    assert b["ess"] == pytest.approx(a["ess"], rel=1e-12)
    assert b["log_j2_mean"] == pytest.approx(a["log_j2_mean"] - 0.7 * 16, rel=1e-12)
    c = orc.jastrow_reweight(X[:, ::-1], v, o=o)
    assert c["mean"] == pytest.approx(a["mean"], rel=1e-13)


def test_repeated_orbital_is_rejected():
    with pytest.raises(ValueError):
        orc.jastrow_reweight([[1, 1]], np.zeros((3, 3)))


def exact_anderson_hubbard(U, V):
    """Exact <D> (double occupancy) and <n_0> (first-site occupation, both spins) in the
    Gutzwiller state, by enumerating every pair of up/down site sets; |phi_0(x)|^2 is
    |det U_up|^2 |det U_down|^2 and J^2 = exp(-V * number of doubly occupied sites)."""
    L, N = U.shape
    sets = list(itertools.combinations(range(L), N))
    p = np.array([np.linalg.det(U[list(S), :]) ** 2 for S in sets])
    mask = [sum(1 << i for i in S) for S in sets]
    d = np.array([[bin(a & b).count("1") for b in mask] for a in mask], dtype=float)
    n0 = np.array([[(a & 1) + (b & 1) for b in mask] for a in mask], dtype=float)
    P = np.outer(p, p)

    def mean(power):
        J2 = np.exp(-power * V * d)
        return (P * J2 * d).sum() / (P * J2).sum(), (P * J2 * n0).sum() / (P * J2).sum()

    return mean(1.0), mean(0.5)


@pytest.mark.parametrize("V", [1.0, 4.0])
def test_exact_enumeration_anderson_hubbard(V):
    L = 6
    U = w.anderson_square(2, 3, 2, 1.0, 0)
    (D_ex, n0_ex), (D_J, n0_J) = exact_anderson_hubbard(U, V)
    B = 8000
    X = np.concatenate([orc.sample(U, B, 11), orc.sample(U, B, 12) + L], axis=1)
    v = dense(w.gutzwiller_csr(L, V), 2 * L)
    q = np.zeros((2 * L, 2 * L))
    q[np.arange(L), np.arange(L) + L] = 1.0          # D = sum_i n_{i up} n_{i down}
    o = np.zeros(2 * L)
    o[0] = o[L] = 1.0                                 # n_0 = n_{0 up} + n_{0 down}
    rD = orc.jastrow_reweight(X, v, q=q)
    rn = orc.jastrow_reweight(X, v, o=o)
    assert abs(rD["mean"] - D_ex) < 5 * rD["stderr"], (rD["mean"], D_ex, rD["stderr"])
    assert abs(rn["mean"] - n0_ex) < 5 * rn["stderr"], (rn["mean"], n0_ex, rn["stderr"])
    # the pin tells J^2 from J: weighting by J alone is far outside the error bar
    assert abs(rD["mean"] - D_J) > 10 * rD["stderr"]


def test_infinite_gutzwiller_penalty_removes_double_occupancy():
    L = 6
    U = w.anderson_square(2, 3, 2, 1.0, 0)
    X = np.concatenate([orc.sample(U, 400, 21), orc.sample(U, 400, 22) + L], axis=1)
    q = np.zeros((2 * L, 2 * L))
    q[np.arange(L), np.arange(L) + L] = 1.0
    r = orc.jastrow_reweight(X, dense(w.gutzwiller_csr(L, 200.0), 2 * L), q=q)
    assert r["mean"] < 1e-80
