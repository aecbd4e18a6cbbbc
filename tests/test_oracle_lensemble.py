"""Pins of the oracle's L-ensemble sampler (main text, text-summarisation example: keep
eigenvector j with probability lambda_j / (lambda_j + 1), then FFS on the kept ones)
against the L-ensemble's definition P(S) = det(C_S) / det(C + I) by brute force, the
per-eigenvector keep frequencies, the expected size, and the special cases that reduce
to plain FFS or to the empty set.  A planted mistake in the keep probability fails the
brute-force test."""
from collections import Counter

import numpy as np
import pytest
from scipy.stats import binomtest, chisquare

from oracle import ffs_oracle as orc
from paper_2109_07358_gb300 import workloads as w


def small_kernel():
    Phi = w.lensemble_quality_features(6, 4, 0.9, seed=3)
    lam, V = w.lensemble_spectrum(Phi)
    return Phi @ Phi.T, lam, V


def draw_sets(V, lam, B, seed=0):
    cnt = Counter()
    for s in range(B):
        cnt[tuple(sorted(orc.lensemble_sample_one(V, lam, seed, s)["x"].tolist()))] += 1
    return cnt


def chi2_pvalue(cnt, P, B):
    keys = [S for S, p in P.items() if p > 1e-12]
    assert sum(cnt.get(S, 0) for S in keys) == B          # nothing outside the support
    obs = np.array([cnt.get(S, 0) for S in keys], dtype=float)
    exp = np.array([P[S] * B for S in keys])
    return chisquare(obs, exp * obs.sum() / exp.sum()).pvalue


@pytest.fixture(scope="module")
def brute():
    C, lam, V = small_kernel()
    P = orc.lensemble_set_probabilities(C)
    assert sum(P.values()) == pytest.approx(1.0, abs=1e-12)
    return C, lam, V, P


def test_brute_force_chi_squared(brute):
    C, lam, V, P = brute
    B = 20000
    assert chi2_pvalue(draw_sets(V, lam, B), P, B) > 0.01


def test_planted_keep_probability_fails(brute, monkeypatch):
    C, lam, V, P = brute
    real = orc.lensemble_selection

    def wrong(lam_, seed, sample):          # keeps with lambda / (lambda + 2) instead
        return real(np.asarray(lam_) / 2.0, seed, sample)

    monkeypatch.setattr(orc, "lensemble_selection", wrong)
    B = 20000
    assert chi2_pvalue(draw_sets(V, lam, B), P, B) < 1e-6


def test_keep_frequencies_and_size():
    lam = np.array([0.05, 0.4, 1.0, 3.0, 30.0])
    B = 4000
    kept = np.zeros(lam.size)
    for s in range(B):
        kept[orc.lensemble_selection(lam, 7, s)] += 1
    for j, lj in enumerate(lam):
        assert binomtest(int(kept[j]), B, lj / (lj + 1)).pvalue > 1e-3
    # pairs of decisions are independent: joint frequency of keeping 1 and 2
    both = sum(1 for s in range(B) if {1, 2} <= set(orc.lensemble_selection(lam, 7, s).tolist()))
    assert binomtest(both, B, (0.4 / 1.4) * 0.5).pvalue > 1e-3


def test_all_kept_reduces_to_plain_ffs():
    U = w.haar(10, 4, seed=1, complex_=False)
    lam = np.full(4, 1e20)                    # lambda / (lambda + 1) rounds to 1
    for s in range(5):
        a = orc.lensemble_sample_one(U, lam, 5, s)
        b = orc.sample_one(U, 5, s)
        assert np.array_equal(a["kept"], np.arange(4))
        assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["m_full"], b["m"])


def test_nothing_kept_is_empty():
    U = w.haar(10, 4, seed=1, complex_=False)
    r = orc.lensemble_sample_one(U, np.array([0.0, -1e-17, 0.0, 0.0]), 0, 0, record=True)
    assert r["x"].size == 0 and r["kept"].size == 0 and r["probs"].shape == (0, 10)


def test_one_body_density_is_the_marginal_kernel_diagonal():
    # P(y in S) = K_yy with K = C (C + I)^-1 = sum_j lambda_j / (lambda_j + 1) u_j u_j^T
    Phi = w.lensemble_quality_features(8, 3, 1.2, seed=5)
    lam, V = w.lensemble_spectrum(Phi)
    C = Phi @ Phi.T
    K = C @ np.linalg.inv(C + np.eye(8))
    B = 6000
    occ = np.zeros(8)
    for s in range(B):
        occ[orc.lensemble_sample_one(V, lam, 2, s)["x"]] += 1
    for y in range(8):
        assert binomtest(int(occ[y]), B, K[y, y]).pvalue > 1e-4
