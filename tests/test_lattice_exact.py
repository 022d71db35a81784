"""Pins of the oracle's RD3Q81 velocity set (Sec. III, Table "tab:weights") against facts
the paper fixes, checked in exact arithmetic.

* the trace conditions <w, c^2n> = (2n+1)!! theta0^n (Sec. III, Eq. (condRed1)) hold as
  polynomial identities in theta0 for n <= 4, and at the printed theta0 for n = 5;
* the isotropy conditions of Table "tab:isotropy_cond" hold;
* the anisotropic parts of the 4th, 6th, once-contracted 8th and thrice-contracted 10th
  order weighted moment tensors vanish (the definition of isotropy, App. A);
* the RD3Q81 column of the printed moment-error table is reproduced
  (tests/golden/rd3q81_moment_errors.txt).

A mistyped table coefficient, a missing or duplicated velocity, or a wrong shell radius
breaks at least one of these.
"""

from fractions import Fraction
from math import prod

import numpy as np
import pytest
import sympy as sp
from mpmath import mp, mpf

from oracle import rd3q81 as O

t = sp.Symbol("t")


def _exact_lattice():
    """(h vectors, sympy weights as polynomials in t) from the oracle's own shell table."""
    lat = O.velocity_set()
    wpoly = {}
    for name, gen, coeffs, den in O._SHELLS:
        wpoly[name] = sum(sp.Rational(c, den) * t ** k for k, c in coeffs.items())
    ws = [None] + [wpoly[n] for n in lat.shell[1:]]
    ws[0] = sp.expand(1 - sum(ws[1:]))
    return lat, ws


def _moment(lat, ws, fn):
    return sp.expand(sum(w * fn(*(sp.Rational(int(x), 2) for x in h)) for w, h in zip(ws, lat.h)))


def test_velocity_count_and_shells():
    lat = O.velocity_set()
    assert lat.q == 81
    assert len({tuple(h) for h in lat.h}) == 81
    counts = {}
    for s in lat.shell:
        counts[s] = counts.get(s, 0) + 1
    assert counts == {"rest": 1, "SC-1": 6, "SC-2": 6, "SC-3": 6, "SC-4": 6, "FCC-1": 12,
                      "FCC-2": 12, "BCC-1/2": 8, "BCC-1": 8, "BCC-3/2": 8, "BCC-5/2": 8}
    # every shell is closed under c -> -c
    hs = {tuple(h) for h in lat.h}
    assert all(tuple(-x for x in h) in hs for h in hs)


def test_traces_exact():
    lat, ws = _exact_lattice()
    for n, dfact in enumerate([1, 3, 15, 105, 945]):
        m = _moment(lat, ws, lambda x, y, z: (x * x + y * y + z * z) ** n)
        assert sp.simplify(m - dfact * t ** n) == 0, n
    # n = 5 holds only at theta0: the remainder is a polynomial whose root is theta0.
    m10 = _moment(lat, ws, lambda x, y, z: (x * x + y * y + z * z) ** 5) - 10395 * t ** 5
    mp.dps = 60
    val = sp.lambdify(t, m10, "mpmath")(mpf(O.THETA0_TEXT))
    assert abs(val) < 1e-22
    # ... and theta0 is a simple root (so the printed digits pin it).
    d = sp.lambdify(t, sp.diff(m10, t), "mpmath")(mpf(O.THETA0_TEXT))
    assert abs(d) > 1.0


def test_isotropy_table_conditions():
    """Table "tab:isotropy_cond": sums over SC (S), FCC (F), BCC (B) shells of w_shell a^k,
    a = the shell's nonzero velocity component.  The once-contracted 8th-order row is
    printed with -384 for the BCC term; the per-shell identities printed just above it
    (BCC: 24 * 16 delta) give +384, and only that reading holds -- see the reading list."""
    mp.dps = 60
    t0 = mpf(O.THETA0_TEXT)
    sums = {"SC": {}, "FCC": {}, "BCC": {}}
    for name, gen, coeffs, den in O._SHELLS:
        a = mpf(max(abs(g) for g in gen)) / 2
        wv = sum(mpf(c) * t0 ** k for k, c in coeffs.items()) / den
        typ = name.split("-")[0]
        for k in (4, 6, 8, 10):
            sums[typ][k] = sums[typ].get(k, 0) + wv * a ** k
    S, F, B = sums["SC"], sums["FCC"], sums["BCC"]
    conds = {
        "4th": 2 * S[4] - 4 * F[4] - 16 * B[4],
        "6th a": 2 * S[6] - 52 * F[6] + 128 * B[6],
        "6th b": 4 * F[6] - 16 * B[6],
        "8th a (sign read +384)": 2 * S[8] - 104 * F[8] + 384 * B[8],
        "8th b": 8 * F[8] - 48 * B[8],
        "10th": 2 * S[10] - 32 * F[10] - 432 * B[10],
    }
    for k, v in conds.items():
        assert abs(v) < 1e-20, (k, v)
    # the row as printed does not hold
    assert abs(2 * S[8] - 104 * F[8] - 384 * B[8]) > 1.0


def test_anisotropic_parts_vanish_exactly():
    lat, ws = _exact_lattice()
    c2 = lambda x, y, z: x * x + y * y + z * z
    checks = [
        # 4th order: <cx^4> = 3 <cx^2 cy^2>
        (lambda x, y, z: x ** 4, lambda x, y, z: 3 * x * x * y * y),
        # 6th order
        (lambda x, y, z: x ** 6, lambda x, y, z: 15 * x * x * y * y * z * z),
        (lambda x, y, z: x ** 4 * y * y, lambda x, y, z: 3 * x * x * y * y * z * z),
        # once-contracted 8th
        (lambda x, y, z: c2(x, y, z) * x ** 6, lambda x, y, z: 15 * c2(x, y, z) * x * x * y * y * z * z),
        (lambda x, y, z: c2(x, y, z) * x ** 4 * y * y, lambda x, y, z: 3 * c2(x, y, z) * x * x * y * y * z * z),
    ]
    for a, b in checks:
        assert sp.simplify(_moment(lat, ws, a) - _moment(lat, ws, b)) == 0
    # thrice-contracted 10th: holds at theta0 (mod the trace polynomial)
    d = _moment(lat, ws, lambda x, y, z: c2(x, y, z) ** 3 * x ** 4) - \
        _moment(lat, ws, lambda x, y, z: 3 * c2(x, y, z) ** 3 * x * x * y * y)
    mp.dps = 60
    assert abs(sp.lambdify(t, d, "mpmath")(mpf(O.THETA0_TEXT))) < 1e-22
    # odd moments vanish by symmetry
    assert _moment(lat, ws, lambda x, y, z: x) == 0
    assert _moment(lat, ws, lambda x, y, z: x ** 3 * y * y) == 0


def test_float_weights_match_exact():
    lat = O.velocity_set()
    for wf, we in zip(lat.w, lat.w_exact):
        assert abs(wf - float(we)) <= 1e-17
    assert np.all(lat.w > 0)
    assert abs(lat.w.sum() - 1.0) < 1e-15
    t0 = lat.theta0
    for n, dfact in enumerate([1, 3, 15, 105, 945, 10395]):
        assert abs(lat.w @ lat.c2 ** n / (dfact * t0 ** n) - 1) < 1e-13


def _dfact(k):
    return prod(range(k - 1, 0, -2)) if k > 0 else 1


def _mb_monomial(ex, ey, ez, t0):
    """Maxwell-Boltzmann moment <c_x^ex c_y^ey c_z^ez> at temperature t0 (unit density)."""
    if ex % 2 or ey % 2 or ez % 2:
        return 0.0
    return _dfact(ex) * _dfact(ey) * _dfact(ez) * t0 ** ((ex + ey + ez) // 2)


def _expand_c2(c2pow, ex, ey, ez):
    """(c_x^2 + c_y^2 + c_z^2)^c2pow c_x^ex c_y^ey c_z^ez as a list of (coef, ex, ey, ez)."""
    x, y, z = sp.symbols("x y z")
    poly = sp.Poly(sp.expand((x ** 2 + y ** 2 + z ** 2) ** c2pow * x ** ex * y ** ey * z ** ez), x, y, z)
    return [(int(c), *m) for m, c in zip(poly.monoms(), poly.coeffs())]


def _golden():
    rows = []
    with open(__file__.replace("test_lattice_exact.py", "golden/rd3q81_moment_errors.txt")) as fh:
        for line in fh:
            if line.strip() and not line.lstrip().startswith("#"):
                c2p, ex, ey, ez, val, dec = line.split()
                rows.append((int(c2p), int(ex), int(ey), int(ez), float(val), int(dec)))
    return rows


@pytest.mark.parametrize("row", _golden())
def test_printed_moment_error_column(row):
    """Table "tab:mometnssbasicmodels", RD3Q81 column: percentage error of non-imposed
    weighted moments against Maxwell-Boltzmann.  Printed values are truncated to their
    decimals, so the computed value must lie within one unit of the last printed digit."""
    c2p, ex, ey, ez, printed, dec = row
    lat = O.velocity_set()
    t0 = lat.theta0
    terms = _expand_c2(c2p, ex, ey, ez)
    m_lat = sum(k * float(lat.w @ (lat.c[:, 0] ** a * lat.c[:, 1] ** b * lat.c[:, 2] ** c))
                for k, a, b, c in terms)
    m_mb = sum(k * _mb_monomial(a, b, c, t0) for k, a, b, c in terms)
    err = (m_lat / m_mb - 1.0) * 100.0
    tol = 1e-9 if dec <= 0 else 10.0 ** (-dec) + 1e-9
    assert abs(err - printed) <= tol, (row, err)
