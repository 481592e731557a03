"""The float-pair (double-float) arithmetic the FP32-pipe kernels use, restated
in numpy float32 and checked against exact rational arithmetic: the accuracy
the kernels' comments claim (an FP64 value split into two floats to about
2^-48; Dot2 sums of m products within a few units of m 2^-48 of
sum |x_k y_k|, against m 2^-53 for an FP64 dot product; the rational
Jacobi rotation orthogonal within a few units of 2^-46 whatever its angle).  This pins the
schemes, not the CUDA code (the GPU parity tests compare that with the
oracle)."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def split(x):
    """x (float64) -> (hi, lo) floats: hi = fl32(x), lo = fl32(x - hi)."""
    hi = f32(x)
    return hi, f32(np.float64(x) - np.float64(hi))


def two_prod(a, b):
    """a b = p + e exactly for floats (the FMA of the kernels: the error of a
    float product is a float, and the float64 product of two floats is exact)."""
    p = f32(a * b)
    e = f32(np.float64(a) * np.float64(b) - np.float64(p))
    return p, e


def two_sum(a, b):
    s = f32(a + b)
    bp = f32(s - a)
    e = f32(f32(a - f32(s - bp)) + f32(b - bp))
    return s, e


def dot2(xs, ys):
    """Dot2 of pairs (Ogita, Rump, Oishi): the running pair (a1, a2)."""
    a1, a2 = f32(0), f32(0)
    for (x1, x2), (y1, y2) in zip(xs, ys):
        p, pe = two_prod(x1, y1)
        q = f32(np.float64(x1) * np.float64(y2) + np.float64(x2) * np.float64(y1) + np.float64(pe))
        a1, te = two_sum(a1, p)
        a2 = f32(a2 + f32(te + q))
    return Fraction(float(a1)) + Fraction(float(a2))


def test_split_is_accurate_to_pair_precision():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(20000) * np.exp2(rng.integers(-50, 50, 20000))
    for v in x:
        hi, lo = split(v)
        err = abs(Fraction(float(v)) - Fraction(float(hi)) - Fraction(float(lo)))
        assert err <= Fraction(2) ** -48 * abs(Fraction(float(v)))


def test_dot2_sum_within_its_bound():
    rng = np.random.default_rng(2)
    for trial in range(40):
        m = int(rng.integers(1, 200))
        x = rng.standard_normal(m) * (10.0 ** rng.uniform(-3, 3, m))
        y = rng.standard_normal(m)
        if trial % 4 == 0:  # heavy cancellation: y chosen so that the sum nearly vanishes
            y[-1] = -float(np.dot(x[:-1], y[:-1])) / x[-1]
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y))
        absum = sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(x, y))
        got = dot2([split(a) for a in x], [split(b) for b in y])
        # per term: the splits of both operands, the dropped x2 y2 and the
        # rounding of the first-order terms (a few units of 2^-48 |x y|); over
        # the sum: the float accumulation of the low part, at most about
        # m 2^-48 sum |x y| (an FP64 dot product: m 2^-53)
        assert abs(got - exact) <= (6 * m + 8) * Fraction(2) ** -48 * absum, \
            (m, float(abs(got - exact) / absum))


def test_rational_rotation_is_orthogonal_for_any_angle():
    rng = np.random.default_rng(3)
    tan_pi8 = float(np.tan(np.pi / 8))
    for u in np.concatenate([rng.uniform(-tan_pi8, tan_pi8, 2000), [0.0, 1e-20, -1e-8, tan_pi8]]):
        u = f32(u)
        q, qe = two_prod(u, u)                      # u^2 exactly
        dh, dl = two_sum(f32(1), q)
        dl = f32(dl + qe)                           # 1 + u^2
        nh, nl = two_sum(f32(1), -q)
        nl = f32(nl - qe)                           # 1 - u^2
        r1 = f32(1) / dh
        r1 = f32(r1 + r1 * f32(f32(1) - dh * r1))   # a Newton step on the float reciprocal
        res = f32(np.float64(1) - np.float64(dh) * np.float64(r1) - np.float64(dl) * np.float64(r1))
        rl = f32(r1 * res)
        rh = f32(r1 + rl)
        r = (rh, f32(rl - f32(rh - r1)))

        def mul(a, b):
            p, e = two_prod(a[0], b[0])
            e = f32(np.float64(a[0]) * np.float64(b[1]) + np.float64(a[1]) * np.float64(b[0]) + np.float64(e))
            h = f32(p + e)
            return h, f32(e - f32(h - p))
        c = mul((nh, nl), r)
        s = mul((f32(2 * u), f32(0)), r)
        cf = Fraction(float(c[0])) + Fraction(float(c[1]))
        sf = Fraction(float(s[0])) + Fraction(float(s[1]))
        # the reciprocal to about 2^-47 and the two pair products to 2^-48:
        # c^2 + s^2 = 1 within a few units of 2^-46
        assert abs(cf * cf + sf * sf - 1) <= Fraction(2) ** -44, float(u)
