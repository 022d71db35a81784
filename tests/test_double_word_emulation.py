"""The double-word (float + float) arithmetic that the FP32-storage kernels use where FP32 is not
precise enough -- the moment read-back and the FP64-quality moments of the step -- emulated
operation by operation in numpy float32 (IEEE round to nearest, like the kernels' __f*_rn
intrinsics) and checked against FP64 on the host:

* TwoSum and TwoProd are error-free: hi + lo equals the exact sum / product;
* the cascaded sums of the step (Sum2 and Dot2 of Ogita, Rump and Oishi), over the 81 stored FP32
  populations of random sites, give rho, rho u and <f, c^2> equal to their FP64 sums;
* the Newton-refined reciprocal and the products used to form u and theta stay within a few units
  of 2^-48 relative.

The GPU side of the same arithmetic is pinned in tests/test_gpu_moments_dw.py."""

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


def test_cascaded_moments_equal_fp64_sums():
    """The step's site_moments_dw over the +/- pairs: sums and differences by TwoSum, products by the
    exact floats c^2 and c_a / 2, every rounding error collected in a second float."""
    lat = O.velocity_set()
    h, w, q = lat.h, lat.w, lat.q
    opp = [int(np.flatnonzero(np.all(h == -h[i], axis=1))[0]) for i in range(q)]
    rest = int(np.flatnonzero(np.all(h == 0, axis=1))[0])
    pairs, seen = [], {rest}
    for i in range(q):
        if i not in seen:
            pairs.append((i, opp[i]))
            seen |= {i, opp[i]}
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(200):
        f = (w * (1 + 0.3 * rng.uniform(-1, 1, q))).astype(f32)
        acc = {k: [f32(0), f32(0)] for k in ("e", "x", "y", "z")}
        pr, qr = f[rest], f32(0)

        def add(key, a, v):
            p, qq = acc[key]
            hh, hl = two_prod(f32(a), v[0])
            t0, t1 = two_sum(p, hh)
            acc[key] = [t0, f32(qq + f32(t1 + fma(f32(a), v[1], hl)))]

        for i, j in pairs:
            s, d = two_sum(f[i], f[j]), two_sum(f[i], f32(-f[j]))
            t0, t1 = two_sum(pr, s[0])
            pr, qr = t0, f32(qr + f32(t1 + s[1]))
            add("e", (h[i] ** 2).sum() / 4.0, s)
            for a, key in enumerate("xyz"):
                if h[i][a]:
                    add(key, 0.5 * h[i][a], d)
        got = [val(fast_two_sum(pr, qr))] + [val(two_sum(*acc[k])) for k in "xyz"] + [val(fast_two_sum(*acc["e"]))]
        fd, c = f.astype(np.float64), h / 2.0
        ref = [fd.sum()] + [(c[:, a] * fd).sum() for a in range(3)] + [((c ** 2).sum(1) * fd).sum()]
        scale = [fd.sum()] + [np.abs(c[:, a] * fd).sum() for a in range(3)] + [((c ** 2).sum(1) * fd).sum()]
        worst = max(worst, max(abs(g - r) / s for g, r, s in zip(got, ref, scale)))
    assert worst <= 4 * 2.0 ** -53, worst


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
