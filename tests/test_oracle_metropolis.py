"""Pins of the oracle's large-L Metropolis sampler (Supplementary Section S-7).

* A short chain follows the Metropolis transition law exactly: for N = 1 (one column,
  weights |U_y|^2, two sites of weight 0) the site after m_cond updates is distributed as
  pi_0 K^m_cond, with pi_0 uniform and K the uniform-proposal Metropolis kernel of the
  stated acceptance rule (chi-squared; a chain that ends on a weight-0 site raises, and
  those cases are counted against the law's mass there).  The same samples reject the
  law of the inverted acceptance ratio.
* A long chain reproduces the exact distribution |det U_S|^2 (brute force, chi-squared).
"""
from collections import Counter

import numpy as np
import pytest
from scipy.stats import chisquare

from oracle import ffs_oracle as orc
from paper_2109_07358_gb300 import workloads as w


def transition(p, inverted=False):
    """Metropolis kernel with uniform proposals over the L sites: a move y0 -> y is accepted
    with min(1, p_y / p_y0) (any p_y > 0 from p_y0 = 0; never into p_y = 0)."""
    L = p.size
    K = np.zeros((L, L))
    for y0 in range(L):
        for y in range(L):
            if y == y0:
                continue
            if p[y] == 0:
                a = 0.0
            elif p[y0] == 0:
                a = 1.0
            else:
                a = min(1.0, (p[y0] / p[y]) if inverted else (p[y] / p[y0]))
            K[y0, y] = a / L
        K[y0, y0] = 1.0 - K[y0].sum()
    return K


def test_short_chain_follows_the_transition_law():
    L, M, B = 8, 3, 20000
    u = np.array([0.5, 0.0, 1.0, 0.3, 0.0, 0.9, 0.2, 0.6])
    U = (u / np.linalg.norm(u))[:, None]
    p = U[:, 0] ** 2
    counts = np.zeros(L + 1)                    # last bin: chain ended on a weight-0 site
    for s in range(B):
        try:
            counts[int(orc.sample_one_metropolis(U, M, 4, s)["x"][0])] += 1
        except FloatingPointError:
            counts[L] += 1
    pi = np.full(L, 1.0 / L) @ np.linalg.matrix_power(transition(p), M)
    exp = np.append(pi[p > 0], pi[p == 0].sum()) * B
    obs = np.append(counts[:L][p > 0], counts[L] + counts[:L][p == 0].sum())
    assert counts[:L][p == 0].sum() == 0       # never placed on a weight-0 site
    assert chisquare(obs, exp).pvalue > 0.01
    wrong = np.full(L, 1.0 / L) @ np.linalg.matrix_power(transition(p, inverted=True), M)
    exp_w = np.append(wrong[p > 0], wrong[p == 0].sum()) * B
    assert chisquare(obs, exp_w).pvalue < 1e-6


@pytest.mark.parametrize("complex_", [False, True])
def test_long_chain_reaches_the_exact_distribution(complex_):
    U = w.haar(6, 2, seed=3, complex_=complex_)
    P = orc.set_probabilities(U)
    B = 3000
    cnt = Counter(tuple(sorted(orc.sample_one_metropolis(U, 40, 1, s)["x"].tolist())) for s in range(B))
    keys = list(P)
    obs = np.array([cnt.get(k, 0) for k in keys])
    exp = np.array([P[k] * B for k in keys])
    assert obs.sum() == B
    assert chisquare(obs, exp).pvalue > 0.01
