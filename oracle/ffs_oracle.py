"""Plain CPU oracle for fast fermion sampling (FFS), arXiv 2109.07358.

THIS IS TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
CPU-baseline leg of the benchmark may import it.  The product path (the CUDA library
and its Python binding) never calls it and shares no code with it.

It is written for a reader checking it against the paper, not for speed: FP64 /
complex128 NumPy, one sample at a time, the steps in the paper's order.

Problem (Eq. 1): draw an ordered N-tuple x = (x_1..x_N), x_j in {0..L-1} (0-based
here; the paper is 1-based), from P(x) = |det U_{x,n}|^2 / N!, U an L x N matrix with
U^dagger U = 1.

Method (main text around Eq. 2 and Eq. 3, Supplementary Section S-1):
  1. draw m, a uniformly random permutation of the N columns;
  2. for k = 1..N draw x_k from P(x_k | x_1..x_{k-1}; m), which is proportional
     to |u_{x_k}^T h|^2, where u_y = U[y, (m_1..m_k)] is a k-dim row vector and h is
     the k-dim normal vector orthogonal to u_{x_1}..u_{x_{k-1}} (Eq. 3);
  3. h comes from Gaussian elimination carried out on the base rows in the full
     N-dimensional space, each new base row being eliminated against the earlier
     ones, followed by back substitution (Section S-1);
  4. the inner products u_y^T h for all sites y give the weights (Section S-1: the
     2Lk operations of step k).

Readings of points the paper leaves open:
  * m is drawn per sample (the identity of Eq. 2 averages over all permutations;
    a fixed column order is biased).
  * The normal vector is h = (h_1..h_{k-1}, 1): its normalisation cancels in the
    conditional, so the last component is fixed to 1.
  * Weights are computed for all L sites and set to exactly 0 on sites already
    drawn (they are 0 in exact arithmetic).
  * Inverse CDF: with C_y the running sum of the weights in site order and
    Z = C_{L-1}, x_k = min{ y : C_y > u Z }; if rounding leaves no such y, the last
    site with a nonzero weight is taken.
  * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed lo32, seed hi32),
    counter = (block, stream, sample lo32, sample hi32).  Stream 0 feeds a
    Fisher-Yates shuffle of (0..N-1): block j serves shuffle steps i = N-1-2j (words
    0, 1) and i = N-2-2j (words 2, 3), each taking r = word_a * 2^32 + word_b and
    swapping m[i] with m[(r * (i+1)) >> 64].  Stream 1 block k gives the uniform of
    step k (0-based): u = ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53.

What pins each part (none compares the oracle with itself):
  * philox4x32_10: the published known-answer vectors (tests/golden).
  * permutation, site_uniform: uniformity over S_4 (chi-squared), the N = 1 and N = 2
    shuffles worked out by hand, 53-bit uniforms in [0, 1) (Kolmogorov-Smirnov).
  * inverse_cdf: hand-made edge cases (zero weights, boundaries, the largest uniform,
    the rounding fallback).
  * sample_one / chain_probability: Eq. 2 by exact enumeration (the average over all N!
    column orders equals |det U_x|^2 / N! for every ordered x, real and complex, up to
    L = 8, N = 4); orders uniform given the set (chi-squared); the
    conditional of every step against its determinant definition; the prefix marginal
    (N-k)!/N! det K_XX of marginal sampling; per-step invariants (Z = |h|^2, zero weight
    on drawn sites, prod |s_k|^2 = |det U_x|^2); N = 1 (Born rule), N = L, U = [I; 0]
    (uniform orders); block-diagonal U (independent blocks); brute force over the 495
    sets of the 12-site chain (chi-squared); one-body and pair densities; the double
    well's deterministic stages and its Bernoulli case.  Planted slips (a transposed
    operand, a sign, >= in the draw, an off-by-one shuffle) fail these pins.
  * the L-ensemble, Metropolis and reweighting functions further down: pinned in their
    own test files (brute-force subset laws, the exact short-chain transition law,
    exact enumeration of small Anderson-Hubbard systems).
  * sample, sample_parallel: loops over sample_one (no arithmetic of their own).
  * target_ordered, conditional_by_determinants, set_probabilities, one_body_density,
    pair_density: the definitions written out (determinants, K = U U^dagger); the tests
    cross-check them with independent determinant loops and Cauchy-Binet.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.linalg import solve_triangular

MASK32 = 0xFFFFFFFF
_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
STREAM_PERM = 0
STREAM_SITE = 1


# --------------------------------------------------------------------------------------
# Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw, SC'11).
# --------------------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Ten Philox4x32 rounds; the key is bumped by the Weyl constants between rounds."""
    c0, c1, c2, c3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _PHILOX_W0) & MASK32
            k1 = (k1 + _PHILOX_W1) & MASK32
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0, p1 & MASK32, (p0 >> 32) ^ c3 ^ k1, p0 & MASK32)
    return c0, c1, c2, c3


def _key(seed: int):
    seed = int(seed)
    return (seed & MASK32, (seed >> 32) & MASK32)


def _ctr(block: int, stream: int, sample: int):
    sample = int(sample)
    return (int(block) & MASK32, stream, sample & MASK32, (sample >> 32) & MASK32)


def permutation(seed: int, sample: int, N: int) -> np.ndarray:
    """The column order m of one sample (0-based), Fisher-Yates from Philox stream 0."""
    m = list(range(N))
    i = N - 1
    block = 0
    while i >= 1:
        w = philox4x32_10(_ctr(block, STREAM_PERM, sample), _key(seed))
        for hi, lo in ((w[0], w[1]), (w[2], w[3])):
            if i < 1:
                break
            r = (hi << 32) | lo
            j = (r * (i + 1)) >> 64
            m[i], m[j] = m[j], m[i]
            i -= 1
        block += 1
    return np.array(m, dtype=np.int64)


def site_uniform(seed: int, sample: int, k: int) -> float:
    """The uniform in [0, 1) used to draw x_k (k 0-based), 53 bits, Philox stream 1."""
    w = philox4x32_10(_ctr(k, STREAM_SITE, sample), _key(seed))
    return float(((w[0] >> 5) << 26) + (w[1] >> 6)) * 2.0**-53


# --------------------------------------------------------------------------------------
# The draw (main text after Eq. 2; tie rule as stated in the module header)
# --------------------------------------------------------------------------------------
def inverse_cdf(p: np.ndarray, u: float) -> int:
    C = np.cumsum(p)
    t = u * C[-1]
    hit = np.nonzero(C > t)[0]
    if hit.size:
        return int(hit[0])
    return int(np.nonzero(p > 0)[0][-1])


# --------------------------------------------------------------------------------------
# One sample, step by step (Eq. 2, Eq. 3, Section S-1)
# --------------------------------------------------------------------------------------
def sample_one(U, seed: int = 0, sample: int = 0, n_steps: int | None = None, m=None,
               force_x=None, record: bool = False):
    """Draw one configuration.

    U        L x N orbitals (float64 or complex128), U^dagger U = 1.
    n_steps  number of fermions to place (N by default; fewer gives the marginal of the
             first n_steps positions, the paper's marginal-sampling case).
    m        column order; drawn from Philox(seed, sample) when None.
    force_x  teacher forcing: x_k is taken from force_x instead of being drawn (the
             weights are still computed), used to compare conditionals step by step.
    record   also return, per step, the normalised conditional over all L sites, the
             normaliser Z_k, the pivot s_k = u_{x_k}^T h and the uniform u_k.

    Returns a dict with 'x' (ordered, int64), 'm', and when record is set 'probs'
    (n_steps x L), 'Z', 's', 'u', 'logp' (log of the chain's probability of x given m),
    'hnorm2' (|h|^2 per step).
    """
    U = np.asarray(U)
    L, N = U.shape
    K = N if n_steps is None else int(n_steps)
    dtype = np.result_type(U.dtype, np.float64)
    m = permutation(seed, sample, N) if m is None else np.asarray(m, dtype=np.int64)
    Ut = U[:, m].astype(dtype)            # row y restricted to the first k columns is u_y
    E = np.zeros((N, N), dtype)           # base rows after elimination, full N-dim space
    x: list[int] = []
    rec = {"probs": [], "Z": [], "s": [], "u": [], "hnorm2": []}
    logp = 0.0
    for k in range(K):                    # k base rows x_0..x_{k-1} are fixed
        if k >= 1:
            # Eliminate the newest base row against the earlier ones (Section S-1):
            # subtract the combination c of earlier echelon rows that zeroes its first
            # k-1 entries, i.e. solve c E[:k-1, :k-1] = r[:k-1] (forward substitution).
            r = Ut[x[k - 1], :].copy()
            if k >= 2:
                c = solve_triangular(E[: k - 1, : k - 1], r[: k - 1], trans="T", lower=False)
                r = r - c @ E[: k - 1, :]
                r[: k - 1] = 0.0
            E[k - 1, :] = r
        # Normal vector h in k+1 dims (Eq. 3): last entry 1, back substitution on the
        # upper-triangular echelon rows for the first k entries.
        h = np.zeros(k + 1, dtype)
        h[k] = 1.0
        if k:
            h[:k] = solve_triangular(E[:k, :k], -E[:k, k], lower=False)
        # Inner products u_y^T h for every site y (Section S-1).
        v = Ut[:, : k + 1] @ h
        p = np.abs(v) ** 2
        if x:
            p[np.array(x)] = 0.0
        u = site_uniform(seed, sample, k)
        if force_x is not None:
            xk = int(force_x[k])
        else:
            xk = inverse_cdf(p, u)
        Z = float(np.cumsum(p)[-1])
        if record:
            rec["probs"].append(p / Z)
            rec["Z"].append(Z)
            rec["s"].append(v[xk])
            rec["u"].append(u)
            rec["hnorm2"].append(float(np.sum(np.abs(h) ** 2)))
        logp += math.log(p[xk] / Z) if p[xk] > 0 else -math.inf
        x.append(xk)
    out = {"x": np.array(x, dtype=np.int64), "m": m}
    if record:
        out["probs"] = np.array(rec["probs"])
        out["Z"] = np.array(rec["Z"])
        out["s"] = np.array(rec["s"])
        out["u"] = np.array(rec["u"])
        out["hnorm2"] = np.array(rec["hnorm2"])
        out["logp"] = logp
    return out


def sample(U, B: int, seed: int = 0, first_sample_index: int = 0, n_steps: int | None = None):
    """B configurations, sample b keyed by (seed, first_sample_index + b); B x n_steps int64."""
    U = np.asarray(U)
    K = U.shape[1] if n_steps is None else n_steps
    out = np.zeros((B, K), dtype=np.int64)
    for b in range(B):
        out[b] = sample_one(U, seed, first_sample_index + b, n_steps=n_steps)["x"]
    return out


def _sample_range(args):
    U, seed, lo, hi, n_steps = args
    return [sample_one(U, seed, s, n_steps=n_steps)["x"] for s in range(lo, hi)]


def sample_parallel(U, B: int, seed: int = 0, first_sample_index: int = 0, n_steps=None,
                    workers: int | None = None):
    """``sample`` over a spawn-started process pool (one single-threaded worker per core)."""
    import multiprocessing as mp
    import os

    workers = workers or os.cpu_count() or 1
    workers = max(1, min(workers, B))
    bounds = np.linspace(first_sample_index, first_sample_index + B, workers + 1).astype(int)
    jobs = [(U, seed, int(bounds[i]), int(bounds[i + 1]), n_steps) for i in range(workers)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_single_thread) as pool:
        parts = pool.map(_sample_range, jobs)
    return np.array([x for part in parts for x in part], dtype=np.int64)


def _single_thread():
    import os

    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    try:
        from threadpoolctl import threadpool_limits

        threadpool_limits(1)
    except Exception:
        pass


# --------------------------------------------------------------------------------------
# Definitional tiers for tiny sizes
# --------------------------------------------------------------------------------------
def conditional_by_determinants(U, m, x_prefix) -> np.ndarray:
    """Unnormalised conditional of step k = len(x_prefix) straight from its definition
    (Eq. 2): |det U[(x_prefix, y), (m_1..m_{k+1})]|^2 for every site y."""
    U = np.asarray(U)
    L = U.shape[0]
    k = len(x_prefix)
    cols = np.asarray(m)[: k + 1]
    p = np.zeros(L)
    for y in range(L):
        rows = list(x_prefix) + [y]
        p[y] = abs(np.linalg.det(U[np.ix_(rows, cols)])) ** 2
    return p


def chain_probability(U, m, x) -> float:
    """Probability that the chain with column order m produces the ordered tuple x."""
    return math.exp(sample_one(U, m=m, force_x=x, record=True)["logp"])


def target_ordered(U, x) -> float:
    """Eq. 1: |det U_{x,n}|^2 / N! for an ordered tuple x."""
    U = np.asarray(U)
    N = U.shape[1]
    return abs(np.linalg.det(U[np.asarray(x), :])) ** 2 / math.factorial(N)


def set_probabilities(U) -> dict:
    """Brute force over all C(L, N) site sets S: P(S) = |det U_S|^2 (sums to 1 by
    Cauchy-Binet when U^dagger U = 1)."""
    U = np.asarray(U)
    L, N = U.shape
    return {S: abs(np.linalg.det(U[list(S), :])) ** 2 for S in itertools.combinations(range(L), N)}


def one_body_density(U) -> np.ndarray:
    """rho(y) = sum_n |U_{y n}|^2, the expected occupation of site y (sums to N)."""
    return np.sum(np.abs(np.asarray(U)) ** 2, axis=1)


def pair_density(U) -> np.ndarray:
    """rho2(y, z) = rho(y) rho(z) - |G(y, z)|^2 with G = U U^dagger (y != z): the
    probability that both y and z are occupied."""
    U = np.asarray(U)
    G = U @ U.conj().T
    rho = np.real(np.diag(G))
    R = np.outer(rho, rho) - np.abs(G) ** 2
    np.fill_diagonal(R, 0.0)
    return R


# --------------------------------------------------------------------------------------
# Slater-Jastrow reweighting (Supplementary Section S-5).
#
# |psi_J> = J |phi_0> with J = exp(-1/2 sum_ij v_ij n_i n_j) diagonal in the configuration
# basis, so <psi_J|O|psi_J> / <psi_J|psi_J> becomes a ratio of free-fermion averages,
# <J^2 o_L>_0 / <J^2>_0, where o_L(x) = <x|O|psi_J> / <x|psi_J>.  For an observable
# diagonal in the configuration basis o_L(x) is its value on x; the ones handled here are
# o_L(x) = sum_i o_i n_i + sum_ij q_ij n_i n_j.
def occupations(X, n_orb: int) -> np.ndarray:
    """B x n_orb matrix of the occupation numbers n_i (0 or 1) of each configuration."""
    X = np.asarray(X, dtype=np.int64)
    n = np.zeros((X.shape[0], n_orb))
    n[np.arange(X.shape[0])[:, None], X] = 1.0
    if np.any(n.sum(axis=1) != X.shape[1]):
        raise ValueError("a configuration names an orbital twice")
    return n


def jastrow_log_weight(X, v) -> np.ndarray:
    """log J^2(x) = -sum_ij v_ij n_i n_j for each configuration (v dense, n_orb x n_orb)."""
    v = np.asarray(v, dtype=np.float64)
    n = occupations(X, v.shape[0])
    return -np.sum((n @ v) * n, axis=1)


def diagonal_observable(X, n_orb: int, o=None, q=None) -> np.ndarray:
    """o_L(x) = sum_i o_i n_i + sum_ij q_ij n_i n_j for each configuration."""
    n = occupations(X, n_orb)
    val = np.zeros(n.shape[0])
    if o is not None:
        val = val + n @ np.asarray(o, dtype=np.float64)
    if q is not None:
        val = val + np.sum((n @ np.asarray(q, dtype=np.float64)) * n, axis=1)
    return val


def jastrow_reweight(X, v, o=None, q=None) -> dict:
    """The reweighting estimate of <O> in the Jastrow state from free-fermion samples X.

    With weights w_b = J^2(x_b) (scaled by exp(-max log J^2), which cancels):
      mean         sum_b w_b o_L(x_b) / sum_b w_b               = <J^2 o_L>_0 / <J^2>_0
      log_j2_mean  log( (1/B) sum_b J^2(x_b) )                  = log <J^2>_0
      ess          (sum_b w_b)^2 / sum_b w_b^2                  (effective sample size)
      stderr       sqrt( sum_b w_b^2 (o_L(x_b) - mean)^2 ) / sum_b w_b
                   (first-order error of a ratio of sample means)
    plus the per-sample log J^2 and o_L."""
    v = np.asarray(v, dtype=np.float64)
    logj2 = jastrow_log_weight(X, v)
    obs = diagonal_observable(X, v.shape[0], o, q)
    mx = logj2.max()
    w = np.exp(logj2 - mx)
    sw = w.sum()
    mean = float((w * obs).sum() / sw)
    return {
        "mean": mean,
        "log_j2_mean": float(mx + math.log(sw / len(w))),
        "ess": float(sw * sw / (w * w).sum()),
        "stderr": float(math.sqrt(((w * (obs - mean)) ** 2).sum()) / sw),
        "logj2": logj2,
        "obs": obs,
    }


# --------------------------------------------------------------------------------------
# L-ensemble DPP (main text, text-summarisation example): the correlation matrix
# C = sum_j lambda_j u_j u_j^T; each eigenvector u_j is kept with probability
# lambda_j / (lambda_j + 1), and the kept ones form the U of Eq. 1, sampled by FFS with
# N = the number kept.
# Reading: the keep decision of eigenvector j of sample s uses its own uniform, Philox
# stream 2, block j, built like the site uniforms (53 bits); u < lambda / (lambda + 1)
# keeps it (never for lambda <= 0).  The kept columns, in ascending order, are the U of
# that sample, whose column order m is then drawn as for any other U (stream 0, with N =
# the number kept).
STREAM_SELECT = 2


def select_uniform(seed: int, sample: int, j: int) -> float:
    """The uniform in [0, 1) that decides whether eigenvector j is kept (Philox stream 2)."""
    w = philox4x32_10(_ctr(j, STREAM_SELECT, sample), _key(seed))
    return float(((w[0] >> 5) << 26) + (w[1] >> 6)) * 2.0**-53


def lensemble_selection(lam, seed: int, sample: int) -> np.ndarray:
    """Indices (ascending) of the eigenvectors kept by sample `sample`."""
    keep = []
    for j, lj in enumerate(np.asarray(lam, dtype=np.float64)):
        p = lj / (lj + 1.0) if lj > 0 else 0.0
        if select_uniform(seed, sample, j) < p:
            keep.append(j)
    return np.array(keep, dtype=np.int64)


def lensemble_sample_one(V, lam, seed: int = 0, sample: int = 0, force_x=None, record: bool = False):
    """One L-ensemble draw: the eigenvectors V[:, j] are kept as decided by
    ``lensemble_selection``, then ``sample_one`` runs on U = V[:, kept] (its own column
    order m over the kept columns).  Adds 'kept' (eigenvector indices) and 'm_full' (the
    column order in V's columns: kept[m]) to the returned dict; an empty selection gives
    an empty x."""
    V = np.asarray(V)
    kept = lensemble_selection(lam, seed, sample)
    if kept.size == 0:
        out = {"x": np.zeros(0, dtype=np.int64), "m": np.zeros(0, dtype=np.int64), "logp": 0.0}
        if record:
            out["probs"] = np.zeros((0, V.shape[0]))
    else:
        out = sample_one(V[:, kept], seed, sample, force_x=force_x, record=record)
    out["kept"] = kept
    out["m_full"] = kept[out["m"]]
    return out


def lensemble_set_probabilities(C) -> dict:
    """Brute force over every subset S of the L items: P(S) = det(C_S) / det(C + I), the
    L-ensemble with kernel C (sums to 1; the empty set has det = 1)."""
    C = np.asarray(C, dtype=np.float64)
    L = C.shape[0]
    Z = np.linalg.det(C + np.eye(L))
    out = {}
    for n in range(L + 1):
        for S in itertools.combinations(range(L), n):
            out[S] = (np.linalg.det(C[np.ix_(S, S)]) if n else 1.0) / Z
    return out


# --------------------------------------------------------------------------------------
# Large-L / continuous-model variant (Supplementary Section S-7): x_k is drawn by a
# Metropolis chain over sites, each move accepted with the ratio
# |u_{y'}^T h|^2 / |u_y^T h|^2, instead of from all L conditional weights.
# Readings (the section leaves them open): the discrete update proposes a uniform site;
# the chain of step k starts at a uniform site; a move is accepted when
# u * w(current) < w(proposed), which is the ratio rule for w(current) > 0 and accepts any
# site with weight when the chain sits on a drawn site (weight 0); m_cond updates per
# step.  Random numbers: Philox stream 3, block k (m_cond + 1) + t for iteration t
# (t = 0 gives the starting site): words 0, 1 -> site floor(r L / 2^64) of r = w0 2^32 + w1;
# words 2, 3 -> the 53-bit uniform, built like the site uniforms.
STREAM_MCMC = 3


def metropolis_randoms(seed: int, sample: int, k: int, t: int, L: int, m_cond: int):
    """(site, uniform) of iteration t of the chain of step k."""
    w = philox4x32_10(_ctr(k * (m_cond + 1) + t, STREAM_MCMC, sample), _key(seed))
    r = (w[0] << 32) | w[1]
    u = float(((w[2] >> 5) << 26) + (w[3] >> 6)) * 2.0**-53
    return (r * L) >> 64, u


def sample_one_metropolis(U, m_cond: int, seed: int = 0, sample: int = 0, n_steps: int | None = None,
                          record: bool = False):
    """One configuration with the large-L draw of Section S-7.  The column order and the
    elimination are those of ``sample_one``; the weight of a site y at step k is
    w(y) = |u_y^T h|^2 (0 on drawn sites), evaluated only where the chain looks.

    Returns 'x' and 'm'; with record, per step 'margin': the smallest relative gap
    |u w(current) - w(proposed)| / max(w(current), w(proposed)) over the chain's
    decisions (how close a decision came to flipping), and 'w_final' (weight of x_k)."""
    U = np.asarray(U)
    L, N = U.shape
    K = N if n_steps is None else int(n_steps)
    dtype = np.result_type(U.dtype, np.float64)
    m = permutation(seed, sample, N)
    Ut = U[:, m].astype(dtype)
    E = np.zeros((N, N), dtype)
    x: list[int] = []
    margins, finals = [], []
    for k in range(K):
        if k >= 1:       # elimination of the newest base row, as in sample_one
            r = Ut[x[k - 1], :].copy()
            if k >= 2:
                c = solve_triangular(E[: k - 1, : k - 1], r[: k - 1], trans="T", lower=False)
                r = r - c @ E[: k - 1, :]
                r[: k - 1] = 0.0
            E[k - 1, :] = r
        h = np.zeros(k + 1, dtype)
        h[k] = 1.0
        if k:
            h[:k] = solve_triangular(E[:k, :k], -E[:k, k], lower=False)
        taken = set(x)

        def weight(y):
            return 0.0 if y in taken else float(abs(Ut[y, : k + 1] @ h) ** 2)

        cur, _ = metropolis_randoms(seed, sample, k, 0, L, m_cond)
        wc = weight(cur)
        margin = math.inf
        for t in range(1, m_cond + 1):
            y, u = metropolis_randoms(seed, sample, k, t, L, m_cond)
            wy = weight(y)
            scale = max(wc, wy)
            if scale > 0:
                margin = min(margin, abs(u * wc - wy) / scale)
            if u * wc < wy:
                cur, wc = y, wy
        if wc <= 0.0:
            raise FloatingPointError(f"sample {sample}, step {k}: the chain found no site with weight")
        margins.append(margin)
        finals.append(wc)
        x.append(int(cur))
    out = {"x": np.array(x, dtype=np.int64), "m": m}
    if record:
        out["margin"] = np.array(margins)
        out["w_final"] = np.array(finals)
    return out
