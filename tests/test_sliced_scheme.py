"""The arithmetic of the sliced dense product, checked exactly on the CPU.

The tensor-core product cuts FP64 entries into balanced base-256 digits: for
a 128-wide chunk of a row of A (or of a column of X) with exponent e (every
|x| < 2^e), round(x 2^(55-e))
= sum_s d_s 2^(8(6-s)) with d_0 in [-128, 128] and d_1..d_6 in [-128, 127],
so x ~ 2^(e-7) sum_s d_s 2^(-8s).  These tests restate that decomposition
with Python integers and fractions (no floating point) and check the facts the
kernel relies on: digit ranges (8 significant bits: exact in bf16), the
rounding error 2^(e-56), the bound 7 * 128 * 2^14 < 2^24 on a chunk's level
sums (exact fp32 accumulation), and the product error bound that the GPU test
asserts, n 2^-50 max|A_i.| max|X_.j|.  The planes of A are stored as bytes
d + 128 under a margin exponent that keeps the leading digit in [-128, 127],
and widened to fp16 on the GPU: both are checked here as well.
"""
import math
from fractions import Fraction

import numpy as np

KS = 7
FRAC = 8 * (KS - 1) + 7  # 55


def exponent(values):
    """e with |x| < 2^e for all x (from the largest exponent field)."""
    m = max(abs(v) for v in values)
    if m == 0.0:
        return -1021
    return math.frexp(m)[1]  # m = f 2^e, 0.5 <= f < 1


def digits(x, e):
    v = round(Fraction(x) * 2 ** (FRAC - e))
    d = [0] * KS
    for s in range(KS - 1, 0, -1):
        lo = v & 0xFF
        dd = (lo ^ 0x80) - 0x80
        d[s] = dd
        v = (v - dd) >> 8
    d[0] = v
    return d


def value(d, e):
    return sum(Fraction(d[s]) * Fraction(2) ** (e - 7 - 8 * s) for s in range(KS))


def test_digit_ranges_and_rounding_error():
    rng = np.random.default_rng(0)
    for trial in range(200):
        row = rng.standard_normal(16) * 2.0 ** rng.integers(-40, 40)
        if trial % 7 == 0:
            row[3] = -np.abs(row).max()  # extreme entry, negative
        e = exponent(row)
        for x in row:
            d = digits(float(x), e)
            assert -128 <= d[0] <= 128
            assert all(-128 <= ds <= 127 for ds in d[1:])
            # every digit has at most 8 significant bits (exact in bf16)
            assert all(abs(ds) < 2 ** 8 + 1 for ds in d)
            err = abs(value(d, e) - Fraction(float(x)))
            assert err <= Fraction(2) ** (e - 56)


def test_extreme_digit_plus_128():
    """An entry just below 2^e rounds its first digit up to 128."""
    e = 3
    x = math.ldexp(1.0, e) * (1 - 2.0 ** -53)
    d = digits(x, e)   # x 2^(55-e) = 2^55 - 4: digits 128, 0, ..., 0, -4
    assert d[0] == 128 and d[1:] == [0] * (KS - 2) + [-4]
    assert value(d, e) == Fraction(x)


def exponent_margin(values):
    """The exponent the A planes use: one more than `exponent` when the
    largest |x| has its top six mantissa bits set (is within 2^-6 of the next
    power of two in its binade), so that every |x| < 2^e (1 - 2^-7)."""
    m = max(abs(v) for v in values)
    if m == 0.0:
        return -1021
    f, e = math.frexp(m)               # m = f 2^e, 0.5 <= f < 1
    top6 = int(f * 2 ** 7) & 0x3F      # mantissa bits 1..6 after the leading one
    return e + 1 if top6 == 0x3F else e


def stored_bytes(d):
    """The A planes' bytes: the digits of v as bytes of v + 128 (1 + 256 + ...)."""
    v = sum(d[s] * 256 ** (KS - 1 - s) for s in range(KS))
    u = v + sum(128 * 256 ** k for k in range(KS))
    assert u >= 0
    return [(u >> (8 * (KS - 1 - s))) & 0xFF for s in range(KS)], u >> (8 * KS)


def test_margin_exponent_puts_every_digit_in_a_byte():
    """With the margin exponent the leading digit stays in [-128, 127], so the
    seven digits of A are the seven bytes of v + 128 (1 + 256 + ... + 256^6)
    with no carry out of the top byte, each byte minus 128 giving its digit."""
    rng = np.random.default_rng(3)
    rows = [rng.standard_normal(16) * 2.0 ** rng.integers(-30, 30) for _ in range(200)]
    for k in range(60):  # largest entries just below a power of two
        r = rng.standard_normal(16)
        r[k % 16] = math.ldexp(1.0, k - 30) * (1 - 2.0 ** -(1 + k % 53))
        rows.append(r)
    for row in rows:
        e = exponent_margin(row)
        assert max(abs(x) for x in row) < 2.0 ** e * (1 - 2.0 ** -7)
        for x in row:
            d = digits(float(x), e)
            assert all(-128 <= ds <= 127 for ds in d)
            b, carry = stored_bytes(d)
            assert carry == 0 and [bb - 128 for bb in b] == d
            assert abs(value(d, e) - Fraction(float(x))) <= Fraction(2) ** (e - 56)


def test_widening_a_byte_to_fp16_is_exact():
    """The product widens a stored byte b = d + 128 to fp16 by placing b in the
    mantissa of 1024 + b and subtracting 1152 in fp16: exact for every byte."""
    b = np.arange(256)
    x = (np.float16(1024) + b.astype(np.float16)).astype(np.float16)
    # the bit pattern 0x6400 | b is 1024 + b
    assert np.array_equal(x.view(np.uint16), (0x6400 | b).astype(np.uint16))
    d = (x - np.float16(1152)).astype(np.float16)
    assert np.array_equal(d.astype(np.int64), b - 128)


def test_level_sums_fit_fp32():
    """Worst case of a level sum over one 128-wide chunk: 7 pairs of digits at
    magnitude 128: every partial sum is an integer below 2^24."""
    worst = 7 * 128 * 128 * 128
    assert worst < 2 ** 24


def sliced_product_exact(A, X):
    """The kernel's arithmetic with exact integers: exponents of A per (row,
    128-column chunk) and of X per (128-row chunk, column), level sums of pairs
    s + t <= 6 over each chunk, the int64 fold at resolution 2^-36 (levels 5, 6
    rounded half up), the shift to the row's and column's largest exponents,
    the sum over chunks."""
    n, p = X.shape
    chunks = [(c0, min(n, c0 + 128)) for c0 in range(0, n, 128)]
    eA = [[exponent(A[i, c0:c1]) for (c0, c1) in chunks] for i in range(n)]
    eX = [[exponent(X[c0:c1, j]) for j in range(p)] for (c0, c1) in chunks]
    dA = [[digits(float(A[i, k]), eA[i][k // 128]) for k in range(n)] for i in range(n)]
    dX = [[None] * p for _ in range(n)]
    for ci, (c0, c1) in enumerate(chunks):
        for k in range(c0, c1):
            for j in range(p):
                dX[k][j] = digits(float(X[k, j]), eX[ci][j])
    Y = np.zeros((n, p), dtype=object)
    for i in range(n):
        amax = max(eA[i])
        for j in range(p):
            emax = max(eX[ci][j] for ci in range(len(chunks)))
            acc = 0
            for ci, (c0, c1) in enumerate(chunks):
                L = [0] * KS
                for k in range(c0, c1):
                    for s in range(KS):
                        for t in range(KS - s):
                            L[s + t] += dA[i][k][s] * dX[k][j][t]
                assert all(abs(v) < 2 ** 24 for v in L)
                v = 0
                for lvl in range(KS):
                    sh = 36 - 8 * lvl
                    v += L[lvl] << sh if sh >= 0 else (L[lvl] + (1 << (-sh - 1))) >> (-sh)
                d = (amax - eA[i][ci]) + (emax - eX[ci][j])
                acc += v if d == 0 else (v + (1 << (d - 1))) >> d
            Y[i, j] = Fraction(acc) * Fraction(2) ** (amax + emax - 14 - 36)
    return Y


def test_sliced_product_error_bound_exact_arithmetic():
    rng = np.random.default_rng(1)
    n, p = 140, 2   # two chunks (128 + 12)
    A = rng.standard_normal((n, n)) * np.exp2(rng.uniform(-10, 10, n))[:, None]
    X = rng.standard_normal((n, p)) * np.exp2(rng.uniform(-10, 10, p))[None, :]
    X[:128, 1] *= 2.0 ** -20  # the two chunks of column 1 get different exponents
    A[::3, 128:] *= 2.0 ** 9   # and so do the two column chunks of every third row
    Y = sliced_product_exact(A, X)
    for i in range(0, n, 7):
        for j in range(p):
            exact = sum(Fraction(float(A[i, k])) * Fraction(float(X[k, j])) for k in range(n))
            bound = Fraction(n) * Fraction(2) ** -50 * Fraction(float(np.abs(A[i]).max())) * \
                Fraction(float(np.abs(X[:, j]).max()))
            assert abs(Y[i, j] - exact) <= bound
