"""Oracle pins on special cases whose answer is fixed independently of the sampler:

* block-diagonal U: a determinant of a block-diagonal matrix vanishes unless each block
  contributes as many rows as it has columns, and then it factorises, so the blocks'
  sites are independent projection DPPs (the set law of Eq. 1 for each block alone);
* the double-well chain of the supplementary double-well section: the particle-number
  difference between the wells is 0 in the balanced stage and 2 in the imbalanced one,
  and where the highest orbital is split between the wells the left count is a Bernoulli
  variable whose error over M samples is sqrt(p (1 - p) / M), p being that orbital's
  weight in the left well;
* Eq. 1 is symmetric in the order of x: given the set, the N! orders are uniform;
* Eq. 2 by exact enumeration at (L, N) = (8, 4).

Expected values come from determinants written out here (numpy's det over every
subset), not from the oracle's own set-probability helper.
"""
from collections import Counter
from itertools import combinations, permutations

import numpy as np
from scipy.stats import chisquare

from oracle import ffs_oracle as orc
from paper_2109_07358_gb300 import workloads as w


def _set_law(U):
    L, N = U.shape
    return {S: float(abs(np.linalg.det(U[list(S), :])) ** 2) for S in combinations(range(L), N)}


def test_block_diagonal_blocks_are_independent():
    U1 = w.haar(4, 2, seed=21)             # block 1: sites 0..3, columns 0..1
    U2 = w.haar(5, 2, seed=22)             # block 2: sites 4..8, columns 2..3
    U = np.zeros((9, 4), complex)
    U[:4, :2] = U1
    U[4:, 2:] = U2
    P1, P2 = _set_law(U1), _set_law(U2)
    assert abs(sum(P1.values()) - 1) < 1e-12 and abs(sum(P2.values()) - 1) < 1e-12  # Cauchy-Binet
    M = 6000
    X = orc.sample(U, M, seed=77)
    joint = Counter()
    for x in X:
        S = sorted(int(v) for v in x)
        left = tuple(v for v in S if v < 4)
        right = tuple(v - 4 for v in S if v >= 4)
        assert len(left) == 2 and len(right) == 2  # every other split has determinant 0
        joint[(left, right)] += 1
    cells = [(a, b) for a in P1 for b in P2]
    exp = np.array([P1[a] * P2[b] * M for a, b in cells])
    obs = np.array([joint.get(c, 0) for c in cells], float)
    # pool the cells expected below 5 into one
    small = exp < 5
    e = np.append(exp[~small], exp[small].sum())
    o = np.append(obs[~small], obs[small].sum())
    p = chisquare(o, e * o.sum() / e.sum()).pvalue
    print(f"block-diagonal U: {len(cells)} joint cells, chi-squared p = {p:.3f}")
    assert p > 1e-3


def _left_count(X, xs):
    return np.array([(xs[np.asarray(x)] < 0).sum() for x in X])


def test_double_well_stages():
    """The supplementary double-well recipe (64 sites evenly on [-2, 2], a = 4096, b = 2,
    hopping pi^2/6, four fermions).  Read with the hopping as the nearest-neighbour
    matrix element, the number difference jumps from 0 to 2 at c = 46.645; the paper
    quotes c = 89.929 for its own discretisation.  Both stages are deterministic in the
    exact law (the tunnelling splitting is below double precision), so every sample must
    show them."""
    for c, n_left in ((20.0, 2), (46.64, 2), (46.65, 1), (89.929, 1)):
        U, xs = w.double_well(c=c)
        K = U @ U.T
        left = xs < 0
        assert abs(np.trace(K[np.ix_(left, left)]) - n_left) < 1e-9
        X = orc.sample(U, 200, seed=5)
        nl = _left_count(X, xs)
        assert (nl == n_left).all(), (c, np.unique(nl))


def test_double_well_bernoulli_error():
    """A symmetric well shallow enough for the tunnelling to split the levels (a = 1,
    c = 0) with an odd filling (N = 3): the third orbital is parity-even, p = 1/2 in the
    left well, and the left count is 1 + Bernoulli(p).  Checked against the exact law of
    the count from all C(64, 3) determinants, and the sample mean against the Bernoulli
    error of the supplementary double-well section."""
    U, xs = w.double_well(L=64, N=3, c=0.0, a=1.0)
    left = xs < 0
    p = float((U[:, -1] ** 2)[left].sum())
    assert abs(p - 0.5) < 1e-8  # parity, up to the eigensolver's mixing of close levels
    law = Counter()
    for S, q in _set_law(U).items():
        law[int(left[list(S)].sum())] += q
    assert abs(law[1] - 0.5) < 1e-8 and abs(law[2] - 0.5) < 1e-8
    assert law[0] < 1e-8 and law[3] < 1e-8
    M = 4000
    nl = _left_count(orc.sample(U, M, seed=9), xs)
    assert set(np.unique(nl)) <= {1, 2}
    eps = np.sqrt(p * (1 - p) / M)
    dev = abs(nl.mean() - 1.5)
    print(f"double well, Bernoulli case: mean left count {nl.mean():.4f} (exact 1.5), "
          f"deviation {dev / eps:.2f} eps, eps = {eps:.4f}")
    assert dev < 5 * eps


def test_orders_are_uniform_given_the_set():
    """Eq. 1 is symmetric in the order of x, so given the set every one of the N! orders
    is equally likely; checked on the most frequent sets of a complex U by chi-squared."""
    U = w.haar(6, 3, seed=31)
    M = 9000
    X = orc.sample(U, M, seed=13)
    by_set = {}
    for x in X:
        t = tuple(int(v) for v in x)
        by_set.setdefault(tuple(sorted(t)), Counter())[t] += 1
    top = sorted(by_set, key=lambda s: -sum(by_set[s].values()))[:4]
    for S in top:
        c = by_set[S]
        obs = np.array([c.get(o, 0) for o in permutations(S)], float)
        assert obs.sum() >= 300
        p = chisquare(obs).pvalue
        print(f"set {S}: {int(obs.sum())} samples over 6 orders, chi-squared p = {p:.3f}")
        assert p > 1e-3


def test_exact_enumeration_L8_N4():
    """Eq. 2 at (L, N) = (8, 4): the chain averaged over all 24 column orders equals
    |det U_x|^2 / N! (determinant written out here) for every one of the 1680 ordered x."""
    from math import factorial

    U = w.haar(8, 4, seed=84)
    perms = list(permutations(range(4)))
    total = 0.0
    for x in permutations(range(8), 4):
        avg = np.mean([orc.chain_probability(U, list(m), list(x)) for m in perms])
        want = abs(np.linalg.det(U[list(x), :])) ** 2 / factorial(4)
        assert abs(avg - want) < 1e-13
        total += avg
    assert abs(total - 1.0) < 1e-12
