"""Pins for the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a published
test vector, an exact identity (Eq. 1 / Eq. 2 by enumeration), a definition (the
determinant form of the conditional), a closed form, or a statistical property of
the target distribution.  A plausible slip in the oracle (a dropped elimination
term, a transposed operand, a wrong sign, an off-by-one in the shuffle, >= instead
of > in the draw) fails at least one of them; ``test_planted_mistakes_are_caught``
plants several such slips and checks that they are caught.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import ffs_oracle as o
from paper_2109_07358_gb300 import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- random numbers
def test_philox_known_answers():
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            t = [int(v, 16) for v in line.split()]
            assert o.philox4x32_10(t[0:4], t[4:6]) == tuple(t[6:10])
            n += 1
    assert n == 3


def test_uniform_is_53_bit_in_unit_interval():
    us = [o.site_uniform(7, s, k) for s in range(50) for k in range(20)]
    for u in us:
        assert 0.0 <= u < 1.0
        assert float(int(u * 2**53)) == u * 2**53
    # uniformity (Kolmogorov-Smirnov)
    assert stats.kstest(us, "uniform").pvalue > 1e-3


def test_permutation_is_uniform_over_S4():
    N = 4
    counts = {}
    n = 24 * 150
    for s in range(n):
        m = tuple(o.permutation(3, s, N))
        assert sorted(m) == list(range(N))
        counts[m] = counts.get(m, 0) + 1
    assert len(counts) == 24
    chi2 = stats.chisquare(list(counts.values()))
    assert chi2.pvalue > 1e-3


def test_permutation_fisher_yates_small_cases():
    # N = 1: nothing to shuffle; N = 2: one swap decided by the top bit of r * 2.
    assert list(o.permutation(0, 0, 1)) == [0]
    for s in range(20):
        w0, w1, _, _ = o.philox4x32_10((0, 0, s, 0), (5, 0))
        swap = ((((w0 << 32) | w1) * 2) >> 64) == 0
        assert list(o.permutation(5, s, 2)) == ([1, 0] if swap else [0, 1])


# ---------------------------------------------------------------- the draw rule
def test_inverse_cdf_edges():
    p = np.array([0.0, 1.0, 0.0, 2.0, 0.0])
    assert o.inverse_cdf(p, 0.0) == 1            # zero-weight sites are never chosen
    assert o.inverse_cdf(p, 1.0 / 3.0 - 1e-12) == 1
    assert o.inverse_cdf(p, 1.0 / 3.0 + 1e-12) == 3
    assert o.inverse_cdf(p, 1.0 - 2.0**-53) == 3  # largest uniform
    assert o.inverse_cdf(np.array([0, 0, 5e-300, 0]), 0.7) == 2
    # u * Z rounding up to Z leaves no y with C_y > t: the last nonzero site is taken
    assert o.inverse_cdf(np.array([1.0, 1.0, 0.0]), 1.0) == 1


# ---------------------------------------------------------------- exactness (Eq. 1, Eq. 2)
@pytest.mark.parametrize("L,N,cplx", [(5, 3, True), (6, 4, False), (5, 2, True), (4, 4, True)])
def test_permutation_average_equals_target(L, N, cplx):
    """Eq. 2: averaging the chain over all N! column orders gives |det U_x|^2/N! (Eq. 1)
    for every ordered x; also the chain is a normalised distribution for each m."""
    U = w.haar(L, N, seed=L * 10 + N, complex_=cplx)
    perms = list(itertools.permutations(range(N)))
    total = 0.0
    for x in itertools.permutations(range(L), N):
        q = [o.chain_probability(U, list(m), list(x)) for m in perms]
        avg = sum(q) / len(perms)
        assert abs(avg - o.target_ordered(U, x)) < 1e-13
        total += avg
    assert abs(total - 1.0) < 1e-12
    for m in perms[:3]:
        s = sum(o.chain_probability(U, list(m), list(x)) for x in itertools.permutations(range(L), N))
        assert abs(s - 1.0) < 1e-12


def test_fixed_column_order_is_biased():
    """The random order is essential: with m fixed the chain misses Eq. 1."""
    U = w.haar(5, 3, seed=1)
    worst = max(abs(o.chain_probability(U, [0, 1, 2], list(x)) - o.target_ordered(U, x))
                for x in itertools.permutations(range(5), 3))
    assert worst > 1e-3


@pytest.mark.parametrize("cplx", [False, True])
def test_conditionals_match_determinant_definition(cplx):
    """Eq. 3 / Section S-1 (normal vector + inner products) reproduce the conditional
    defined by determinants in Eq. 2, at every step."""
    U = w.haar(9, 5, seed=11, complex_=cplx)
    for s in range(4):
        r = o.sample_one(U, seed=2, sample=s, record=True)
        for k in range(5):
            p = o.conditional_by_determinants(U, r["m"], list(r["x"][:k]))
            assert np.max(np.abs(p / p.sum() - r["probs"][k])) < 1e-12


def test_prefix_marginal_is_projection_dpp_marginal():
    """Marginal sampling (stopping after N_< steps): averaged over m, the first k
    positions have probability (N-k)!/N! det K_XX with K = U U^dagger."""
    U = w.haar(5, 3, seed=4)
    L, N = U.shape
    K = U @ U.conj().T
    perms = list(itertools.permutations(range(N)))
    for k in (1, 2):
        for xp in itertools.permutations(range(L), k):
            avg = np.mean([math.exp(o.sample_one(U, m=list(m), force_x=list(xp), n_steps=k,
                                                 record=True)["logp"]) for m in perms])
            want = math.factorial(N - k) / math.factorial(N) * np.linalg.det(K[np.ix_(xp, xp)]).real
            assert abs(avg - want) < 1e-13


# ---------------------------------------------------------------- invariants per step
@pytest.mark.parametrize("cplx", [False, True])
def test_step_invariants(cplx):
    U = w.haar(40, 12, seed=5, complex_=cplx)
    for s in range(3):
        r = o.sample_one(U, seed=9, sample=s, record=True)
        x = r["x"]
        assert len(set(x.tolist())) == 12
        for k in range(12):
            # sum_y |v_y|^2 = |h|^2 = 1 + |w|^2 (U^dagger U = 1), and chosen sites carry 0
            assert abs(r["Z"][k] - r["hnorm2"][k]) < 1e-10 * r["hnorm2"][k]
            assert np.all(r["probs"][k][x[:k]] == 0.0)
            assert abs(r["probs"][k].sum() - 1.0) < 1e-12
        # the pivots multiply to the determinant: prod |s_k|^2 = |det U_{x,n}|^2
        assert abs(np.prod(np.abs(r["s"]) ** 2) - abs(np.linalg.det(U[x, :])) ** 2) < 1e-10 * abs(
            np.linalg.det(U[x, :])) ** 2


# ---------------------------------------------------------------- special cases
def test_single_fermion_is_born_rule():
    U = w.haar(30, 1, seed=3)
    r = o.sample_one(U, record=True)
    assert np.allclose(r["probs"][0], np.abs(U[:, 0]) ** 2, atol=1e-15)


def test_full_filling_and_identity_block():
    U = w.haar(6, 6, seed=2)
    for s in range(5):
        assert sorted(o.sample_one(U, sample=s)["x"].tolist()) == list(range(6))
    U = np.zeros((9, 4))
    U[:4, :4] = np.eye(4)
    orders = {}
    for s in range(24 * 40):
        x = o.sample_one(U, sample=s)["x"]
        assert sorted(x.tolist()) == [0, 1, 2, 3]
        orders[tuple(x)] = orders.get(tuple(x), 0) + 1
    assert len(orders) == 24 and stats.chisquare(list(orders.values())).pvalue > 1e-3


def test_open_chain_closed_form_is_the_eigenbasis():
    L, N = 64, 8
    U = w.open_chain(L, N)
    H = w.open_chain_hamiltonian(L)
    E = -2 * np.cos(np.pi * np.arange(1, N + 1) / (L + 1))
    assert np.allclose(H @ U, U * E, atol=1e-13)
    assert np.allclose(U.T @ U, np.eye(N), atol=1e-13)
    evals = np.linalg.eigvalsh(H)
    assert np.allclose(evals[:N], E, atol=1e-12) and evals[N] > E[-1] + 1e-6


# ---------------------------------------------------------------- brute force (statistics)
def _chi2_pvalue(observed: dict, expected_p: dict, n: int):
    keys = sorted(expected_p, key=lambda s: expected_p[s])
    obs, exp = [], []
    acc_o = acc_e = 0.0
    for s in keys:                       # merge the smallest cells until expected >= 5
        acc_o += observed.get(s, 0)
        acc_e += expected_p[s] * n
        if acc_e >= 5:
            obs.append(acc_o)
            exp.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0:
        obs[-1] += acc_o
        exp[-1] += acc_e
    exp = np.array(exp) * (n / np.sum(exp))
    return stats.chisquare(obs, exp).pvalue


def test_brute_force_chain_L12_N4():
    """All C(12, 4) = 495 sets of the open chain: P(S) = |det U_S|^2 sums to 1
    (Cauchy-Binet), and 10^4 oracle samples pass chi-squared at p > 0.01."""
    U = w.open_chain(12, 4)
    P = o.set_probabilities(U)
    assert len(P) == 495 and abs(sum(P.values()) - 1.0) < 1e-13
    n = 10_000
    X = o.sample(U, n, seed=0)
    counts = {}
    for x in X:
        S = tuple(sorted(x.tolist()))
        counts[S] = counts.get(S, 0) + 1
    assert _chi2_pvalue(counts, P, n) > 0.01


def test_one_body_and_pair_density():
    """Sample occupations against rho(y) = sum_n |U_yn|^2 (sum N) and the pair density
    rho(y) rho(z) - |G(y,z)|^2, G = U U^dagger, as z-scores."""
    U = w.square_lattice(4, 4, 8, seed=1)
    L, N = U.shape
    rho = o.one_body_density(U)
    assert abs(rho.sum() - N) < 1e-12
    R2 = o.pair_density(U)
    n = 3000
    X = o.sample(U, n, seed=1)
    occ = np.zeros((n, L))
    occ[np.arange(n)[:, None], X] = 1
    mean = occ.mean(0)
    z = (mean - rho) / np.sqrt(np.maximum(rho * (1 - rho), 1e-12) / n)
    assert np.max(np.abs(z)) < 4.5
    pair = (occ.T @ occ) / n
    iu = np.triu_indices(L, 1)
    z2 = (pair[iu] - R2[iu]) / np.sqrt(np.maximum(R2[iu] * (1 - R2[iu]), 1e-12) / n)
    assert np.max(np.abs(z2)) < 5.0


# ---------------------------------------------------------------- the pins have teeth
def test_planted_mistakes_are_caught(monkeypatch):
    """Plant slips in a copy of the oracle's arithmetic and check a pin fails."""
    U = w.haar(5, 4, seed=1)
    perms = list(itertools.permutations(range(4)))

    def eq2_error():
        return max(abs(np.mean([o.chain_probability(U, list(m), list(x)) for m in perms])
                       - o.target_ordered(U, x)) for x in itertools.permutations(range(5), 4))

    assert eq2_error() < 1e-13
    real_solve = o.solve_triangular

    # (1) transposed operand in the elimination of the new base row
    def wrong_trans(a, b, trans=0, lower=False, **kw):
        return real_solve(a, b, trans=0, lower=lower, **kw)
    monkeypatch.setattr(o, "solve_triangular", wrong_trans)
    assert eq2_error() > 1e-6
    monkeypatch.setattr(o, "solve_triangular", real_solve)

    # (2) wrong sign in the back substitution of h
    def wrong_sign(a, b, trans=0, lower=False, **kw):
        out = real_solve(a, b, trans=trans, lower=lower, **kw)
        return out if trans == "T" else -out
    monkeypatch.setattr(o, "solve_triangular", wrong_sign)
    assert eq2_error() > 1e-6
    monkeypatch.setattr(o, "solve_triangular", real_solve)

    # (3) >= instead of > in the inverse CDF picks zero-weight sites
    def ge_cdf(p, u):
        C = np.cumsum(p)
        return int(np.nonzero(C >= u * C[-1])[0][0])
    monkeypatch.setattr(o, "inverse_cdf", ge_cdf)
    p = np.array([0.0, 1.0, 0.0, 2.0])
    assert o.inverse_cdf(p, 0.0) != 1
    monkeypatch.undo()

    # (4) Fisher-Yates with an off-by-one range (idx in [0, i) instead of [0, i]) is not uniform
    def fy_offbyone(seed, sample, N):
        m = list(range(N))
        for i in range(N - 1, 0, -1):
            wv = o.philox4x32_10((i, 0, sample, 0), (seed, 0))
            j = ((((wv[0] << 32) | wv[1]) * i) >> 64)
            m[i], m[j] = m[j], m[i]
        return tuple(m)
    seen = {fy_offbyone(3, s, 4) for s in range(2000)}
    assert len(seen) < 24
