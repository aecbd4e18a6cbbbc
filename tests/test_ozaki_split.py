"""The arithmetic argument of the tensor-core trailing update, checked on the CPU with
exact rationals.  The scheme (Ozaki, Ogita, Oishi & Rump 2012) as the kernels use it:
a double-float value x (a pair of FP32 numbers) scaled by a power of two sigma >= |x| is
cut into six 8-bit integer slices by FP32 arithmetic (round to nearest integer, exact
remainder by an error-free sum, multiply by 256); the products of slices a_i b_j with
i + j <= 8 are accumulated per d = i + j in FP32 over K = 64.  The claims:

* every slice is an integer with |a_i| <= 128, so it is exact in BF16;
* the six slices and the remainder add up to x / sigma exactly, and the remainder is
  below 2^-48;
* every FP32 partial sum of one accumulator is an integer below 2^23 (so the tensor-core
  accumulation is exact whatever its order);
* the dropped products (i + j > 8) and the remainders together stay below
  2^-46 sigma_r sigma_c K of the exact product;
* a subnormal maximum takes sigma = 2^-125 and its slices stay finite and exact.

The new rows' kernel slices W0_T more cheaply (three exact digits of the high part, then
the low part folded into the remainder by one FMA) and adds the seven groups with FP32
for the three smallest and lazy error-free sums for the rest; for those the claims are a
remainder of at most 2^-47, a fourth digit of at most 256 (still exact in BF16), group
sums of at most 2^23, and the chunk's product still within 2^-46 sigma sigma K.

The slicing below is an FP32 restatement of the same steps (numpy float32 rounds to
nearest even like the kernels' _rn operations); the expected values are exact rationals.
"""
from fractions import Fraction

import numpy as np
import pytest

F = np.float32
SLICES, DMAX, K = 6, 8, 64


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    e = F(F(a - F(s - bb)) + F(b - bb))
    return s, e


def pow2_scale(mx):
    if not mx > 0:
        return F(1.0), F(1.0)
    _, e = np.frexp(F(mx))
    e = max(int(e), -125)
    return F(np.ldexp(1.0, e)), F(np.ldexp(1.0, -e))


def slices(hi, lo):
    th, tl = F(hi * F(128)), F(lo * F(128))
    out = []
    for _ in range(SLICES):
        a = F(np.rint(th))
        assert F(th - a) + a == th                     # th - a is exact
        rh, rl = two_sum(F(th - a), tl)
        out.append(a)
        th, tl = F(rh * F(256)), F(rl * F(256))
    return out, Fraction(float(th)) + Fraction(float(tl))  # remainder (scaled by 2^55)


def random_df(rng, n, scale=1.0):
    hi = (rng.standard_normal(n) * scale).astype(F)
    lo = (rng.standard_normal(n) * np.abs(hi) * 2.0**-25).astype(F)
    return hi, lo


def exact(hi, lo):
    return Fraction(float(hi)) + Fraction(float(lo))


@pytest.mark.parametrize("scale", [1.0, 1e-20, 1e20])
def test_slices_are_exact_bf16_integers_and_sum_to_x(scale):
    rng = np.random.default_rng(1)
    hi, lo = random_df(rng, 64, scale)
    sigma, inv = pow2_scale(float(np.max(np.abs(hi))))
    assert sigma >= np.max(np.abs(hi))
    for h, l in zip(hi, lo):
        s, rem = slices(F(h * inv), F(l * inv))
        for a in s:
            assert float(a).is_integer() and abs(a) <= 128    # 8 bits and a sign: exact in BF16
        recon = sum(Fraction(int(a)) * Fraction(1, 2 ** (7 + 8 * i)) for i, a in enumerate(s))
        remainder = rem * Fraction(1, 2 ** (7 + 8 * SLICES))
        x = exact(F(h * inv), F(l * inv))
        assert recon + remainder == x                          # an exact decomposition
        assert abs(remainder) <= Fraction(1, 2 ** 48)


def _split_matrix(hi, lo, axis):
    """Per row (axis=1) or column (axis=0) power-of-two scales and slices (integers)."""
    mx = np.max(np.abs(hi), axis=axis)
    n = hi.shape[1 - axis]
    sig = np.zeros(n, object)
    S = np.zeros((SLICES,) + hi.shape, np.int64)
    for r in range(n):
        sg, inv = pow2_scale(float(mx[r]))
        sig[r] = Fraction(float(sg))
        idx = (r, slice(None)) if axis == 1 else (slice(None), r)
        for q, (h, l) in enumerate(zip(hi[idx], lo[idx])):
            s, _ = slices(F(h * inv), F(l * inv))
            for i in range(SLICES):
                if axis == 1:
                    S[i, r, q] = int(s[i])
                else:
                    S[i, q, r] = int(s[i])
    return S, sig


def test_product_accumulators_are_exact_and_truncation_is_bounded():
    rng = np.random.default_rng(2)
    M, T = 6, 5
    Ah, Al = random_df(rng, M * K)
    Bh, Bl = random_df(rng, K * T)
    Ah, Al, Bh, Bl = Ah.reshape(M, K), Al.reshape(M, K), Bh.reshape(K, T), Bl.reshape(K, T)
    Ah[2] *= F(1e-30)                                           # rows and columns of very
    Al[2] *= F(1e-30)                                           # different magnitudes
    Bh[:, 1] *= F(1e12)
    Bl[:, 1] *= F(1e12)
    SA, sr = _split_matrix(Ah, Al, axis=1)
    SB, sc = _split_matrix(Bh, Bl, axis=0)
    for r in range(M):
        for c in range(T):
            acc = Fraction(0)
            for d in range(2, DMAX + 1):
                part = 0
                for i in range(1, SLICES + 1):
                    j = d - i
                    if 1 <= j <= SLICES:
                        for k in range(K):                     # any accumulation order
                            part += int(SA[i - 1, r, k]) * int(SB[j - 1, k, c])
                            assert abs(part) < 2 ** 23        # FP32 holds it exactly
                acc += Fraction(part) * Fraction(1, 2 ** (14 + 8 * (d - 2)))
            got = acc * sr[r] * sc[c]
            want = sum(exact(Ah[r, k], Al[r, k]) * exact(Bh[k, c], Bl[k, c]) for k in range(K))
            assert abs(got - want) <= Fraction(1, 2 ** 46) * sr[r] * sc[c] * K


def test_worst_case_partial_sum_is_below_2_23():
    # the most slice pairs share d = 7 (six pairs); all slices at their bound 128
    pairs = max(sum(1 for i in range(1, SLICES + 1) if 1 <= d - i <= SLICES) for d in range(2, DMAX + 1))
    assert pairs == 6
    assert pairs * K * 128 * 128 < 2 ** 23


def test_subnormal_row_maximum_keeps_finite_exact_slices():
    hi = np.array([F(3e-40), F(-1e-41), F(0.0)], F)           # FP32 subnormals
    assert np.all(np.abs(hi[:2]) < np.finfo(F).tiny)
    sigma, inv = pow2_scale(float(np.max(np.abs(hi))))
    assert sigma == F(2.0**-125) and np.isfinite(inv)
    for h in hi:
        s, rem = slices(F(h * inv), F(0.0))
        recon = sum(Fraction(int(a)) * Fraction(1, 2 ** (7 + 8 * i)) for i, a in enumerate(s))
        assert recon + rem * Fraction(1, 2 ** (7 + 8 * SLICES)) == Fraction(float(h)) / Fraction(float(sigma))
    # without the clamp the inverse scale of a subnormal maximum overflows
    _, e = np.frexp(F(3e-40))
    with np.errstate(over="ignore"):
        assert not np.isfinite(F(np.ldexp(F(1.0), -int(e))))


def slices_fast(hi, lo):
    """The new-row kernel's slicing step: the remainder pair is renormalised with the fast
    two-sum (s = d + tl, e = tl - (s - d)); each step is checked to be error-free."""
    th, tl = F(hi * F(128)), F(lo * F(128))
    out = []
    for _ in range(SLICES):
        a = F(np.rint(th))
        d = F(th - a)
        assert Fraction(float(d)) == Fraction(float(th)) - Fraction(float(a))   # exact difference
        s = F(d + tl)
        e = F(tl - F(s - d))
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(d)) + Fraction(float(tl))  # error-free
        out.append(a)
        th, tl = F(s * F(256)), F(e * F(256))
    return out, Fraction(float(th)) + Fraction(float(tl))


def adversarial_df(rng, n):
    """Double-float values at the edges of the fast two-sum's condition: lo at +-ulp(hi)/2,
    hi with few significant bits or integral after scaling, tiny and zero lo."""
    hi = rng.standard_normal(n).astype(F)
    hi[: n // 4] = np.round(hi[: n // 4] * 64) / 64            # few significant bits
    ulp = np.spacing(np.abs(hi)).astype(F)
    lo = (rng.choice([-0.5, 0.5, 0.25, -0.125, 0.0], n) * ulp).astype(F)
    lo[n // 2: n // 2 + 4] = F(1e-40)                           # subnormal low parts
    return hi, lo


@pytest.mark.parametrize("gen", ["random", "adversarial"])
def test_fast_two_sum_slicing_is_exact(gen):
    rng = np.random.default_rng(7)
    hi, lo = random_df(rng, 256) if gen == "random" else adversarial_df(rng, 256)
    sigma, inv = pow2_scale(float(np.max(np.abs(hi))))
    for h, l in zip(hi, lo):
        s, rem = slices_fast(F(h * inv), F(l * inv))
        for a in s:
            assert float(a).is_integer() and abs(a) <= 128
        recon = sum(Fraction(int(a)) * Fraction(1, 2 ** (7 + 8 * i)) for i, a in enumerate(s))
        remainder = rem * Fraction(1, 2 ** (7 + 8 * SLICES))
        assert recon + remainder == exact(F(h * inv), F(l * inv))
        assert abs(remainder) <= Fraction(1, 2 ** 48)


def test_chunked_new_row_product_error():
    """One 64-row chunk of Y's product sum_j W[j, c] C[i, j] as the kernel forms it: per
    (column, chunk) and (row, chunk) power-of-two scales, six fast-two-sum slices each,
    the 26 products with i + j <= 8 summed in FP32 per group (integers below 2^21), groups
    added with weights 2^(-8(d-2)) and the scales: within 2^-46 sigma_c sigma_i K of the
    exact rational product."""
    rng = np.random.default_rng(11)
    for scale_w, scale_c in ((1.0, 1.0), (30.0, 1e-3), (1e-30, 5.0)):
        wh, wl = random_df(rng, K, scale_w)
        ch, cl = random_df(rng, K, scale_c)
        sw, iw = pow2_scale(float(np.max(np.abs(wh))))
        sc, ic = pow2_scale(float(np.max(np.abs(ch))))
        A = [slices_fast(F(h * iw), F(l * iw))[0] for h, l in zip(wh, wl)]
        Bm = [slices_fast(F(h * ic), F(l * ic))[0] for h, l in zip(ch, cl)]
        total = Fraction(0)
        for d in range(2, DMAX + 1):
            acc = F(0)
            for k in range(K):
                for i in range(1, SLICES + 1):
                    j = d - i
                    if 1 <= j <= SLICES:
                        acc = F(acc + F(A[k][i - 1] * Bm[k][j - 1]))
                        assert float(acc).is_integer() and abs(acc) < 2 ** 21
            total += Fraction(float(acc)) * Fraction(1, 2 ** (8 * (d - 2)))
        approx = total * Fraction(float(sw)) * Fraction(float(sc)) / 2 ** 14
        truth = sum(exact(a, b) * exact(c, e) for a, b, c, e in zip(wh, wl, ch, cl))
        bound = Fraction(float(sw)) * Fraction(float(sc)) * K / 2 ** 46
        assert abs(approx - truth) <= bound, (scale_w, scale_c, float(abs(approx - truth) / bound))


def test_smallest_scale_keeps_the_scaling_finite():
    """A column chunk whose largest entry is far below FP32's normal range takes the floor
    scale sigma = 2^-125; x / sigma is formed first and then multiplied by 2^7, because the
    single factor 2^125 x 2^7 would overflow FP32 (and 0 x inf would turn zero entries into
    NaN).  The slices of such values stay finite, exact and sum to x / sigma."""
    sigma, inv = pow2_scale(1e-40)
    with np.errstate(over="ignore"):
        assert float(inv) == 2.0 ** 125 and not np.isfinite(F(inv * F(128)))   # the factor that overflows
    for h in (F(1e-40), F(0.0), F(-3e-39), F(1.2e-38)):
        th, tl = F(F(h * inv) * F(128)), F(F(F(0.0) * inv) * F(128))
        assert np.isfinite(th) and np.isfinite(tl)
        s, rem = slices_fast(F(h * inv), F(0.0))
        recon = sum(Fraction(int(a)) * Fraction(1, 2 ** (7 + 8 * i)) for i, a in enumerate(s))
        assert recon + rem * Fraction(1, 2 ** (7 + 8 * SLICES)) == Fraction(float(F(h * inv)))


def slices_fold(hi, lo):
    """The new-row kernel's slicing of W0_T (hi, lo already divided by sigma): three digits
    of th = hi 2^7 by exact steps (rint, subtract, times 2^8), then the low part joins the
    remainder in one FMA (th + lo 2^31, a single rounding), then three more digits; the
    remainder after the sixth digit is dropped."""
    th = F(hi * F(128))
    out = []
    for _ in range(3):
        a = F(np.rint(th))
        d = F(th - a)
        assert Fraction(float(d)) == Fraction(float(th)) - Fraction(float(a))   # exact
        out.append(a)
        th = F(d * F(256))
    # FMA: the exact value th + lo 2^31 (exact in float64: both are short dyadic numbers)
    # rounded once to FP32
    th = F(float(th) + float(lo) * 2.0 ** 31)
    for _ in range(3):
        a = F(np.rint(th))
        out.append(a)
        th = F(F(th - a) * F(256))
    return out


def fold_worst_cases(rng, n):
    """Values whose folded sum reaches its bound: hi just below sigma with few significant
    bits (so the remainder after three digits is large) and lo at +-ulp(hi)/2."""
    hi = (rng.uniform(0.5, 1.0, n) * rng.choice([-1.0, 1.0], n)).astype(F)
    hi[: n // 2] = (np.round(hi[: n // 2] * 2.0 ** 23) / 2.0 ** 23).astype(F)
    ulp = np.spacing(np.abs(hi)).astype(F)
    lo = (rng.choice([-0.5, 0.5, 0.499, -0.499], n) * ulp).astype(F)
    return hi, lo


@pytest.mark.parametrize("gen", ["random", "adversarial", "worst"])
def test_folded_slicing_error_and_digit_bounds(gen):
    rng = np.random.default_rng(17)
    if gen == "random":
        hi, lo = random_df(rng, 512)
    elif gen == "adversarial":
        hi, lo = adversarial_df(rng, 512)
    else:
        hi, lo = fold_worst_cases(rng, 512)
    sigma, inv = pow2_scale(float(np.max(np.abs(hi))))
    big = 0.0
    for h, l in zip(hi, lo):
        s = slices_fold(F(h * inv), F(l * inv))
        for i, a in enumerate(s):
            assert float(a).is_integer() and abs(a) <= (256 if i == 3 else 128)   # exact in BF16
        big = max(big, abs(float(s[3])))
        recon = sum(Fraction(int(a)) * Fraction(1, 2 ** (7 + 8 * i)) for i, a in enumerate(s))
        assert abs(recon - exact(F(h * inv), F(l * inv))) <= Fraction(1, 2 ** 47)
    if gen == "worst":
        assert big > 128          # the fourth digit does exceed 128 on these inputs


def test_folded_group_sums_stay_exact():
    # |a_4| <= 256 on the W0_T side only; the worst group sums over a 64-row chunk
    aw = [128, 128, 128, 256, 128, 128]
    bc = [128] * 6
    worst = max(sum(aw[i - 1] * bc[d - i - 1] for i in range(1, 7) if 1 <= d - i <= 6) * K for d in range(2, DMAX + 1))
    assert worst <= 2 ** 23           # integers of at most 2^23: exact in FP32 in any order


def group_sum(G):
    """The epilogue's sum of the seven group accumulators G[d] (d = 2..8, integers): G_8,
    G_7 and G_6 in FP32 (the FMA rounded once), then G_5 .. G_2 by lazy error-free sums,
    then one renormalisation (oz_group_sum, lz_get)."""
    t = F(float(F(G[8])) * 2.0 ** -16)
    t = F(float(G[7]) * 2.0 ** -8 + float(t))                 # fmaf: one rounding
    hi = F(F(float(G[6]) + float(t)) * F(2.0 ** -32))         # one rounding, then exact
    lo = F(0.0)
    for d in range(5, 1, -1):
        x = F(F(G[d]) * F(2.0 ** (-8 * (d - 2))))
        s, e = two_sum(hi, x)
        hi, lo = s, F(lo + e)
    s, e = two_sum(hi, lo)
    return Fraction(float(s)) + Fraction(float(e))


def test_folded_chunk_product_with_group_sum():
    """One 64-row chunk of the new rows' product as the kernel now forms it: W0_T's slices
    by the fold, C's by error-free steps, the 26 group products exact, the groups added by
    group_sum: within 2^-46 sigma_w sigma_c K of the exact rational product."""
    rng = np.random.default_rng(23)
    for trial, (scale_w, scale_c) in enumerate(((1.0, 1.0), (30.0, 1e-3), (1e-30, 5.0), (1.0, 1.0))):
        if trial == 3:
            wh, wl = fold_worst_cases(rng, K)
        else:
            wh, wl = random_df(rng, K, scale_w)
        ch, cl = random_df(rng, K, scale_c)
        sw, iw = pow2_scale(float(np.max(np.abs(wh))))
        sc, ic = pow2_scale(float(np.max(np.abs(ch))))
        A = [slices_fold(F(h * iw), F(l * iw)) for h, l in zip(wh, wl)]
        Bm = [slices_fast(F(h * ic), F(l * ic))[0] for h, l in zip(ch, cl)]
        G = {}
        for d in range(2, DMAX + 1):
            G[d] = sum(int(A[k][i - 1]) * int(Bm[k][d - i - 1]) for k in range(K) for i in range(1, SLICES + 1)
                       if 1 <= d - i <= SLICES)
            assert abs(G[d]) <= 2 ** 23
        approx = group_sum(G) * Fraction(float(sw)) * Fraction(float(sc)) / 2 ** 14
        truth = sum(exact(a, b) * exact(c, e) for a, b, c, e in zip(wh, wl, ch, cl))
        bound = Fraction(float(sw)) * Fraction(float(sc)) * K / 2 ** 46
        assert abs(approx - truth) <= bound, (trial, float(abs(approx - truth) / bound))


def test_group_sum_rounding():
    """The FP32 step of the three smallest groups costs at most 2^-33 of a unit of G_2;
    the lazy sums and the final renormalisation add the double-float rounding, 2^-47 of
    the value.  Cases include cancellation (G_2 = 0, small G_3)."""
    rng = np.random.default_rng(29)
    for t in range(3000):
        G = {d: int(rng.integers(-2 ** 23, 2 ** 23 + 1)) for d in range(2, DMAX + 1)}
        if t % 3 == 1:
            G[2], G[3] = 0, int(rng.integers(-50, 51))
        want = sum(Fraction(G[d]) * Fraction(1, 2 ** (8 * (d - 2))) for d in G)
        assert abs(group_sum(G) - want) <= Fraction(1, 2 ** 33) + abs(want) / 2 ** 47
