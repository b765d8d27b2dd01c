"""CPU check of the arithmetic argument behind the biased double-FP32 accumulator that the
delayed-CGS2 first-pass dot products use (df_acc_biased in the CUDA sources).  Each step is
emulated on FP32 values with exact rational arithmetic and round-to-nearest-even to FP32, in the
kernel's order:
    t = fl(x_h·y_h + s_h)       (one fma)
    q = t - s_h                 (exact: Sterbenz, s_h and t stay within [3M/4, 5M/4])
    s_l = fl(s_l + fl(x_h·y_h - q));  s_l = fl(x_h·y_l + s_l);  s_l = fl(x_l·y_h + s_l)
with s_h starting at the power of two M >= 4·T·max|x_h|·max|y_h| (T products).  Checked: q and the
final s_h - M are exact, and the sum differs from the exact Σ (x_h + x_l)(y_h + y_l) by at most
(3T² + 2T)·2^-47·M: each step rounds the fma remainder once (below 2^-24 ulp(M)) and adds three
terms into s_l, whose size stays below about T·2^-23·M."""
from fractions import Fraction as Fr

import numpy as np


def r32(x: Fr) -> Fr:
    """x rounded to the nearest FP32 number (ties to even), as an exact rational (normal range)."""
    if x == 0:
        return Fr(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fr(2) ** e > a:
        e -= 1
    scale = Fr(2) ** (e - 23)                  # 24-bit significand
    m = a / scale
    q, r = divmod(m.numerator, m.denominator)
    rem = Fr(r, m.denominator)
    if rem > Fr(1, 2) or (rem == Fr(1, 2) and q % 2 == 1):
        q += 1
    return s * q * scale


def split32(v: float):
    h = r32(Fr(v))
    return h, r32(Fr(v) - h)


def pow2_ceil(y: Fr) -> Fr:
    p = Fr(1)
    while p < y:
        p *= 2
    while p / 2 >= y:
        p /= 2
    return p


def biased_sum(terms, M):
    sh, sl = M, Fr(0)
    for xh, xl, yh, yl in terms:
        t = r32(xh * yh + sh)
        q = r32(t - sh)
        assert q == t - sh                       # Sterbenz
        sl = r32(sl + r32(xh * yh - q))
        sl = r32(xh * yl + sl)
        sl = r32(xl * yh + sl)
        sh = t
    d = r32(sh - M)
    assert d == sh - M                           # removing the bias is exact
    return d + sl


def test_biased_accumulator_is_exact_where_claimed_and_within_its_bound():
    rng = np.random.default_rng(7)
    n = 408321
    for trial in range(8):
        T = [8, 30, 46][trial % 3]
        scale = [1.0, 1e3, 1e-3, 37.0][trial % 4]
        v = rng.standard_normal(T) / np.sqrt(n)
        x = rng.standard_normal(T) / np.sqrt(n) * scale
        if trial % 2:
            x[0] *= -50.0                        # one large term, cancelling sums
        terms = [split32(a) + split32(b) for a, b in zip(v, x)]
        vm = max(abs(t[0]) for t in terms)
        xm = max(abs(t[2]) for t in terms)
        M = pow2_ceil(r32(Fr(4.001) * T * vm * xm))
        got = biased_sum(terms, M)
        exact = sum((xh + xl) * (yh + yl) for xh, xl, yh, yl in terms)
        bound = (3 * T * T + 2 * T) * Fr(1, 2 ** 47) * M
        assert abs(got - exact) <= bound, (trial, float(abs(got - exact)), float(bound))


def test_round_to_fp32_matches_numpy():
    rng = np.random.default_rng(3)
    for v in rng.standard_normal(200) * 10.0 ** rng.integers(-20, 20, 200):
        assert r32(Fr(float(v))) == Fr(float(np.float32(v)))
