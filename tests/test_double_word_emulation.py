"""The double-word (float + float) arithmetic that the FP32-storage kernels use where FP32 is not
precise enough -- the moment read-back and the FP64-quality moments of the step -- emulated
operation by operation in numpy float32 (IEEE round to nearest, like the kernels' __f*_rn
intrinsics) and checked against FP64 on the host:

* TwoSum and TwoProd are error-free: hi + lo equals the exact sum / product;
* the step's FP64-quality moments of FP32 populations (exact 64-bit integer sums of the
  populations scaled by 2^K, returned as double words), over random sites of any magnitude, stay
  within (-2^62, 2^62) and equal the exact sums to the FP64 level;
* the Newton-refined reciprocal and the products used to form u and theta stay within a few units
  of 2^-48 relative.

The GPU side of the same arithmetic is pinned in tests/test_gpu_moments_dw.py."""

from fractions import Fraction

import numpy as np

from oracle import rd3q81 as O

f32 = np.float32
EPS2 = 2.0 ** -48


def two_sum(a, b):
    s = f32(a + b)
    bv = f32(s - a)
    return s, f32(f32(a - f32(s - bv)) + f32(b - bv))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def fma(a, b, c):
    """float32 fused multiply-add: the FP64 product of two floats is exact, one rounding."""
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_prod(a, b):
    p = f32(a * b)
    return p, fma(a, b, -p)


def dw_mul(x, y):
    ch, cl = two_prod(x[0], y[0])
    cross = fma(x[1], y[0], f32(x[0] * y[1]))
    return fast_two_sum(ch, f32(cl + cross))


def dw_recip(y):
    t = f32(f32(1.0) / y[0])
    ph, pl = two_prod(y[0], t)
    d = f32(f32(f32(1.0) - ph) - fma(y[1], t, pl))
    return fast_two_sum(t, f32(d * t))


def val(x):
    return np.float64(x[0]) + np.float64(x[1])


def test_error_free_transformations():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        a, b = f32(rng.normal() * 10 ** rng.uniform(-3, 3)), f32(rng.normal() * 10 ** rng.uniform(-3, 3))
        s, e = two_sum(a, b)
        assert np.float64(s) + np.float64(e) == np.float64(a) + np.float64(b)
        p, q = two_prod(a, b)
        assert np.float64(p) + np.float64(q) == np.float64(a) * np.float64(b)


def _f32_of_int(m: int) -> np.float32:
    """The float nearest the integer m (ties to even), as __ll2float_rn rounds."""
    if m == 0:
        return f32(0.0)
    a = abs(m)
    shift = max(a.bit_length() - 24, 0)
    q, r = divmod(a, 1 << shift)
    half = (1 << shift) >> 1
    if shift and (r > half or (r == half and q & 1)):
        q += 1
    return f32(np.ldexp(np.float64(q if m > 0 else -q), shift))


def _fixed_moments(f, h, pairs, rest):
    """The step's site_moments_dw for FP32 storage, step by step: the bound B in FP32 (|f| and
    fused multiply-adds), the exponent K, every population scaled by 2^K and rounded to an integer
    (ties to even, as __float2ll_rn), shell sums weighted by the integers h^2 and |h_a|, and each
    total returned as a double word.  Also returns the largest |partial sum| seen."""
    B = f32(abs(f[rest]))
    for i, j in pairs:
        g = f32(1.0 + (h[i] ** 2).sum())
        B = fma(f32(f32(abs(f[i])) + f32(abs(f[j]))), g, B)
    Bu = f32(B * f32(1.0009765625))
    e = int((np.array(Bu, dtype=f32).view(np.uint32) >> 23) & 0xFF) - 126
    K = min(61 - e, 120)

    def q(v):
        t = np.float64(v) * 2.0 ** K  # f 2^K: exact in FP32, and so in FP64
        # the kernel's conversion: a = rint(t 2^-31), b = t - a 2^31 (an exact float), then
        # rint(t) = a 2^31 + rint(b) from two 32-bit conversions
        a = np.rint(t * 2.0 ** -31)
        b = t - a * 2.0 ** 31
        assert abs(a) <= 2.0 ** 30 and abs(b) <= 2.0 ** 30 and np.float64(f32(b)) == b
        r = int(a) * 2 ** 31 + int(np.rint(b))
        assert r == int(np.rint(t))
        return r

    tot = {"r": q(f[rest]), "e": 0, "x": 0, "y": 0, "z": 0}
    peak = abs(tot["r"])
    shells = {}
    for i, j in pairs:
        shells.setdefault(int((h[i] ** 2).sum()), []).append((i, j))
    for h2, members in shells.items():
        S = {"s": 0, "x": 0, "y": 0, "z": 0}
        k = int(np.abs(h[members[0][0]]).max())
        for i, j in members:
            ip, im = q(f[i]), q(f[j])
            S["s"] += ip + im
            for a, key in enumerate("xyz"):
                if h[i][a]:
                    S[key] += (ip - im) if h[i][a] > 0 else (im - ip)
            peak = max([peak] + [abs(v) for v in S.values()])
        tot["r"] += S["s"]
        tot["e"] += h2 * S["s"]
        for key in "xyz":
            tot[key] += k * S[key]
        peak = max([peak] + [abs(v) for v in tot.values()])

    def dw(m, scale_exp):
        hi = _f32_of_int(m)
        lo = _f32_of_int(m - int(hi))
        return np.ldexp(np.float64(hi), scale_exp) + np.ldexp(np.float64(lo), scale_exp)

    exps = [-K, -K - 1, -K - 1, -K - 1, -K - 2]
    ints = [tot[k] for k in "rxyze"]
    got = [dw(m, x) for m, x in zip(ints, exps)]
    exact_ints = [Fraction(m) * Fraction(2) ** x for m, x in zip(ints, exps)]
    return got, exact_ints, peak, float(B)


def test_fixed_point_moments_equal_fp64_sums():
    """The step's FP64-quality moments for FP32 storage: exact integer sums of the populations
    scaled by 2^K.  Over random FP32 sites -- near equilibrium at densities from 1e-12 to 1e12,
    and far from it with mixed signs -- no partial sum leaves (-2^62, 2^62), and rho, rho u and
    <f, c^2> equal their exact sums within the rounding of the integers (2^-54 B for rho, 2^-51 B
    for <f, c_a> and <f, c^2>, B = sum |f_i| (1 + h_i^2)); the double word then carries the
    integer to 2^-48 of itself."""
    lat = O.velocity_set()
    h, w, q = lat.h, lat.w, lat.q
    opp = [int(np.flatnonzero(np.all(h == -h[i], axis=1))[0]) for i in range(q)]
    rest = int(np.flatnonzero(np.all(h == 0, axis=1))[0])
    pairs, seen = [], {rest}
    for i in range(q):
        if i not in seen:
            pairs.append((i, opp[i]))
            seen |= {i, opp[i]}
    c = h / 2.0
    rng = np.random.default_rng(1)
    worst, rounded = 0.0, 0
    for n in range(300):
        if n % 3 == 2:
            f = (w * rng.normal(0.0, 2.0, q) * 10 ** rng.uniform(-3, 3)).astype(f32)
        else:
            f = (w * (1 + 0.3 * rng.uniform(-1, 1, q)) * 10 ** rng.uniform(-12, 12)).astype(f32)
            if n % 3 == 1:  # some populations far below the rest: their low bits are rounded off
                f[rng.choice(q, 20, replace=False)] *= f32(10.0 ** rng.uniform(-25, -12))
        got, ints, peak, B = _fixed_moments(f, h, pairs, rest)
        assert peak < 2 ** 62, (n, peak)
        F = [Fraction(float(v)) for v in f]
        ref = [sum(F)] + [sum(Fraction(int(h[i, a]), 2) * F[i] for i in range(q)) for a in range(3)]
        ref += [sum(Fraction(int((h[i] ** 2).sum()), 4) * F[i] for i in range(q))]
        bounds = [2.0 ** -54 * B] + [2.0 ** -51 * B] * 3 + [2.0 ** -51 * B]
        for g, m, r, bd in zip(got, ints, ref, bounds):
            err = abs(float(m - r))                       # the integers' rounding
            assert err <= bd, (n, float(r), err, bd)
            assert abs(g - float(m)) <= 2.0 ** -48 * abs(float(m)), (n, g, float(m))  # the double word
            worst = max(worst, err / bd)
            rounded += err > 0
    print("worst error / integer-rounding bound:", worst, "inexact moments:", rounded)
    assert rounded > 0  # the rounding path was exercised


def test_reciprocal_and_products():
    rng = np.random.default_rng(2)
    for _ in range(3000):
        yv = rng.uniform(0.1, 10.0)
        y = fast_two_sum(f32(yv), f32((yv - np.float64(f32(yv)))))
        r = dw_recip(y)
        assert abs(val(r) * val(y) - 1.0) <= 4 * EPS2
        xv = rng.uniform(-3, 3)
        x = fast_two_sum(f32(xv), f32(xv - np.float64(f32(xv))))
        m = dw_mul(x, y)
        assert abs(val(m) - val(x) * val(y)) <= 8 * EPS2 * abs(val(x) * val(y))


def test_offset_moments_near_fp64_sums():
    """The step's site_moments_dw_offset (FP16/BF16 offset storage, d = f/w - 1): per shell the
    offsets are summed by cascaded TwoSum (S_s, and the signed J_a,s over members with h_a != 0),
    each shell sum is multiplied by the shell's weights held as double words (w_s, w_s c_s^2,
    w_s k_s / 2) and the products accumulated the same way.  Over FP16-representable offsets of
    random sites the result equals the FP64 sums rho = 1 + <w, d>, j = <w, d c>,
    <f, c^2> = 3 theta0 + <w, d c^2> to a few units of 2^-48 of their scale."""
    lat = O.velocity_set()
    h, w, q = lat.h, lat.w, lat.q
    opp = [int(np.flatnonzero(np.all(h == -h[i], axis=1))[0]) for i in range(q)]
    rest = int(np.flatnonzero(np.all(h == 0, axis=1))[0])
    c2 = (h.astype(np.float64) ** 2).sum(1) / 4.0
    kmax = np.abs(h).max(axis=1)
    # +/- pairs grouped by shell (shell = (|c|^2, nonzero pattern): the same weight)
    pairs, seen = [], {rest}
    for i in range(q):
        if i not in seen:
            pairs.append((i, opp[i]))
            seen |= {i, opp[i]}
    shells = {}
    for i, j in pairs:
        shells.setdefault(round(w[i], 15), []).append((i, j))

    def split(v):
        hi = f32(v)
        return hi, f32(v - np.float64(hi))

    def acc(pq, v):
        t0, t1 = two_sum(pq[0], v[0])
        return [t0, f32(pq[1] + f32(t1 + v[1]))]

    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(200):
        d = np.float16(rng.normal(size=q) * 10 ** rng.uniform(-3, 0.7, q)).astype(f32)
        tot = {k: [f32(0), f32(0)] for k in ("r", "e", "x", "y", "z")}
        tot["r"] = acc(tot["r"], dw_mul((d[rest], f32(0)), split(w[rest])))
        for members in shells.values():
            i0 = members[0][0]
            S = {k: [f32(0), f32(0)] for k in ("s", "x", "y", "z")}
            for i, j in members:
                s, df = two_sum(d[i], d[j]), two_sum(d[i], f32(-d[j]))
                S["s"] = acc(S["s"], s)
                for a, key in enumerate("xyz"):
                    if h[i][a]:
                        S[key] = acc(S[key], df if h[i][a] > 0 else (f32(-df[0]), f32(-df[1])))
            ws, wc2, whk = split(w[i0]), split(w[i0] * c2[i0]), split(w[i0] * 0.5 * kmax[i0])
            tot["r"] = acc(tot["r"], dw_mul(two_sum(*S["s"]), ws))
            tot["e"] = acc(tot["e"], dw_mul(two_sum(*S["s"]), wc2))
            for key in "xyz":
                tot[key] = acc(tot[key], dw_mul(two_sum(*S[key]), whk))
        got = [1.0 + val(two_sum(*tot["r"]))] + [val(two_sum(*tot[k])) for k in "xyz"] + \
              [3.0 * lat.theta0 + val(two_sum(*tot["e"]))]
        dd, c = d.astype(np.float64), h / 2.0
        ref = [1.0 + (w * dd).sum()] + [(w * c[:, a] * dd).sum() for a in range(3)] + \
              [3.0 * lat.theta0 + (w * c2 * dd).sum()]
        scale = [1.0 + np.abs(w * dd).sum()] + [np.abs(w * c[:, a] * dd).sum() for a in range(3)] + \
                [3.0 * lat.theta0 + np.abs(w * c2 * dd).sum()]
        worst = max(worst, max(abs(g - r) / s for g, r, s in zip(got, ref, scale)))
    assert worst <= 16 * EPS2, worst
