"""The arithmetic that the Lloyd update's exact route rests on, checked on the CPU in IEEE
float32 / float64 (numpy rounds every operation to nearest, as the kernels' __fadd_rn and
fma do), against exact rational arithmetic.

1. The magic-constant split of a value x with 2^-17 <= |x| < 2^5: t = fl(96 + x),
   hi = t - 96, lo = x - hi, u = fl(1.5 * 2^-17 + lo).  Then bits(t) - bits(96) = hi / 2^-17
   and bits(u) - bits(1.5 * 2^-17) = lo / 2^-40 exactly, so sums of the bit patterns taken
   modulo 2^32 count the parts of the exact sum.
2. The quotient of the centroid mean: RN(s / c) from y = RN(1 / c) by q = RN(s y), then two
   corrections q <- RN(q + RN(s - c q) y) with the residual formed by a fused multiply-add
   (Markstein's theorem makes the second one exact).

Neither is the kernel itself (the GPU parity tests compare the centroids bit for bit); these
pin the two identities on many more cases, including ties and binade edges.
"""
from fractions import Fraction

import numpy as np
import pytest

K1 = np.float32(96.0)
K2 = np.float32(1.5 * 2.0 ** -17)


def _split(x):
    x = np.asarray(x, dtype=np.float32)
    t = (K1 + x).astype(np.float32)
    hi = (t - K1).astype(np.float32)
    lo = (x - hi).astype(np.float32)
    u = (K2 + lo).astype(np.float32)
    return t.view(np.uint32), u.view(np.uint32)


def _in_range_values(rng, n):
    e = rng.uniform(-17.0, 5.0, n)
    x = (rng.choice([-1.0, 1.0], n) * 2.0 ** e).astype(np.float32)
    x = x[(np.abs(x) >= 2.0 ** -17) & (np.abs(x) < 32.0)]
    # ties at the 2^-17 grid (lo = +-2^-18), both binade ends of u, the range ends, zeros
    k = rng.integers(0, 2 ** 22, 64)
    ties = ((k * 2.0 ** -17 + 2.0 ** -18) * rng.choice([-1.0, 1.0], 64)).astype(np.float32)
    ties = ties[(np.abs(ties) >= 2.0 ** -17) & (np.abs(ties) < 32.0)]
    edges = np.array([2.0 ** -17, -2.0 ** -17, np.nextafter(np.float32(32), np.float32(0)),
                      -np.nextafter(np.float32(32), np.float32(0)), 3 * 2.0 ** -18, -3 * 2.0 ** -18,
                      5 * 2.0 ** -18, 0.0, -0.0], dtype=np.float32)
    return np.concatenate([x, ties, edges])


def test_split_parts_are_exact():
    rng = np.random.default_rng(1)
    x = _in_range_values(rng, 400_000)
    tb, ub = _split(x)
    hi = tb.astype(np.int64) - int(K1.view(np.uint32))
    lo = ub.astype(np.int64) - int(K2.view(np.uint32))
    assert np.all(np.abs(hi) <= 2 ** 22) and np.all(np.abs(lo) <= 2 ** 22)
    units = x.astype(np.float64) * 2.0 ** 40               # exact: x is a multiple of 2^-40
    assert np.all(units == np.round(units))
    assert np.array_equal(hi * (1 << 23) + lo, units.astype(np.int64))


def test_wrapped_pattern_sums_count_the_exact_sum():
    """Sixteen values per lane and eight lanes per chunk, as in the kernel: the pattern sums
    modulo 2^32, minus the constants once per added value, give the exact sum."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        x = _in_range_values(rng, 400)[:128]
        rng.shuffle(x)
        tb, ub = _split(x)
        th = tl = np.uint32(0)
        with np.errstate(over="ignore"):
            for q in range(0, len(x), 16):              # per lane, then combined
                lane_t = np.uint32(tb[q:q + 16].astype(np.uint64).sum() % (1 << 32))
                lane_u = np.uint32(ub[q:q + 16].astype(np.uint64).sum() % (1 << 32))
                n = len(tb[q:q + 16])
                sh = np.int32(np.uint32((int(lane_t) - n * int(K1.view(np.uint32))) % (1 << 32)).view(np.int32))
                sl = np.int32(np.uint32((int(lane_u) - n * int(K2.view(np.uint32))) % (1 << 32)).view(np.int32))
                th = th + np.uint32(np.int64(sh) % (1 << 32))
                tl = tl + np.uint32(np.int64(sl) % (1 << 32))
        s = int(np.uint32(th).view(np.int32)) * (1 << 23) + int(np.uint32(tl).view(np.int32))
        exact = sum(Fraction(float(v)) for v in x)
        assert Fraction(s, 1 << 40) == exact


def _rn(fr):
    """Round a rational to the nearest double (ties to even), through its exact decimal-free
    numerator/denominator: float(Fraction) rounds correctly."""
    return float(fr)


def _fma(a, b, c):
    return _rn(Fraction(a) * Fraction(b) + Fraction(c))


def _div_rn(s, c, y):
    q = s * y                                              # numpy/Python double: RN
    r = _fma(-q, c, s)
    q = _fma(r, y, q)
    r = _fma(-q, c, s)
    return _fma(r, y, q)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_reciprocal_division_is_correctly_rounded(seed):
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(3000):
        c = int(rng.integers(1, 1 << 18))
        m = int(rng.integers(1, 1 << 53))                  # a sum with at most 53 bits
        s = float(m) * 2.0 ** int(rng.integers(-80, 20))
        cases.append((s, c))
    # quotients close to a midpoint between two doubles: s = c * (q + half an ulp) rounded
    for _ in range(3000):
        c = int(rng.integers(3, 1 << 18))
        q = float(rng.uniform(0.5, 2.0)) * 2.0 ** int(rng.integers(-40, 10))
        mid = Fraction(q) + Fraction(np.spacing(q)) / 2
        s = _rn(mid * c)
        cases.append((s, c))
    for s, c in cases:
        y = 1.0 / c                                        # RN(1 / c)
        assert _div_rn(s, c, y) == _rn(Fraction(s) / c) == s / c
