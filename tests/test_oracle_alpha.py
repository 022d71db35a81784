"""Pins of the oracle's entropic alpha (Sec. II, Eq. (delH)): the nontrivial root of
Delta H(alpha) = H[f + alpha (feq - f)] - H[f], H = <f, log(f/w) - 1>, with feq the exact
entropic equilibrium of f's conserved moments.  Checked against what fixes it, not against its
own formulas:

* Delta H against the definition itself, H evaluated term by term in 50-digit arithmetic
  (mpmath), at several alpha, near and far from equilibrium;
* the root: the 50-digit Delta H changes sign across it;
* the small-deviation limit: alpha -> 2, with alpha - 2 = a3 / (3 a2) + O(eps^2),
  a_n = <f, x^n>, x = (feq - f)/f (the first two terms of the series of Delta H);
* no root where every population stays positive -> alpha = alpha_max, and Delta H < 0 there;
* f = feq -> alpha = 2;
* the discrete H theorem of the whole step: on a periodic grid streaming only permutes
  populations, so with entropic alpha and beta <= 1 the total H never grows; mass, momentum
  and energy stay conserved.
"""

import numpy as np
import pytest

from oracle import rd3q81 as O

mpmath = pytest.importorskip("mpmath")

LAT = O.velocity_set()
T0 = LAT.theta0
CS = np.sqrt(5.0 * T0 / 3.0)


def _pair(n, mach, eps, seed, eta=0.1):
    """(f, feq): f = feq0 * exp(eps * v) around a random state, feq = the exact entropic
    equilibrium of f's own moments."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    u = d * mach * CS * rng.uniform(0.3, 1.0, n)
    rho = rng.uniform(0.7, 1.3, n)
    th = T0 * (1 + eta * rng.uniform(-1, 1, n))
    f0, _, _ = O.entropic_equilibrium(rho, u, th)
    f = f0 * np.exp(eps * rng.uniform(-1, 1, size=f0.shape))
    r, uu, t = O.moments(f)
    feq, _, _ = O.entropic_equilibrium(r, uu, t)
    return f, feq


def _dh_exact(alpha, f, feq):
    """H[f + alpha D] - H[f] from the definition, in 50-digit arithmetic, one site."""
    with mpmath.workdps(50):
        a = mpmath.mpf(alpha)
        tot = mpmath.mpf(0)
        for fi, gi, wi in zip(f, feq, LAT.w):
            fi, gi, wi = mpmath.mpf(fi), mpmath.mpf(gi), mpmath.mpf(wi)
            y = fi + a * (gi - fi)
            hy = (y * (mpmath.log(y / wi) - 1)) if y > 0 else mpmath.mpf(0)
            tot += hy - fi * (mpmath.log(fi / wi) - 1)
        return tot


@pytest.mark.parametrize("mach,eps", [(0.3, 1e-3), (0.5, 3e-2), (1.5, 0.3)])
def test_delta_h_matches_definition(mach, eps):
    f, feq = _pair(3, mach, eps, seed=int(100 * mach + 1e3 * eps))
    D = feq - f
    amax = np.where(D < 0, f / np.where(D < 0, -D, 1.0), np.inf).min(axis=0)
    checked = 0
    for alpha in (0.5, 1.0, 2.0, 2.4):
        got = O.entropic_delta_h(alpha, f, feq)
        for k in range(f.shape[1]):
            if alpha >= amax[k]:          # H is defined only while every population is positive
                continue
            checked += 1
            ref = float(_dh_exact(alpha, f[:, k], feq[:, k]))
            scale = (f[:, k] * ((feq[:, k] - f[:, k]) / f[:, k]) ** 2).sum()   # ~ size of Delta H
            assert abs(got[k] - ref) <= 1e-9 * scale, (alpha, got[k], ref, scale)
    assert checked >= 8


@pytest.mark.parametrize("mach,eps", [(0.0, 1e-4), (0.5, 1e-2), (1.0, 0.1), (2.0, 0.4)])
def test_root_brackets_definition(mach, eps):
    f, feq = _pair(4, mach, eps, seed=7 + int(10 * mach))
    alpha = O.entropic_alpha(f, feq)
    D = feq - f
    amax = np.where(D < 0, f / np.where(D < 0, -D, 1.0), np.inf).min(axis=0)
    roots = 0
    for k in range(f.shape[1]):
        a = alpha[k]
        assert 1.0 < a <= amax[k] * (1 + 1e-14)
        if abs(a - amax[k]) <= 1e-14 * amax[k]:   # no root before the positivity boundary
            assert _dh_exact(a * (1 - 1e-12), f[:, k], feq[:, k]) < 0
            continue
        roots += 1
        assert np.all(f[:, k] + a * D[:, k] > 0)
        # the bracket: 1e-8, widened by the conditioning of the definition on these float64
        # inputs -- <D, log(feq/w)> vanishes only to the rounding of feq, which shifts the
        # root of H[f + alpha D] - H[f] by about alpha |<D, log(feq/w)>| / <f, x^2>
        with mpmath.workdps(50):
            off = abs(sum((mpmath.mpf(g) - mpmath.mpf(h)) * mpmath.log(mpmath.mpf(g) / mpmath.mpf(w))
                          for h, g, w in zip(f[:, k], feq[:, k], LAT.w)))
        a2 = (f[:, k] * ((feq[:, k] - f[:, k]) / f[:, k]) ** 2).sum()
        d = 1e-8 + 10.0 * a * float(off) / a2
        lo, hi = _dh_exact(a * (1 - d), f[:, k], feq[:, k]), _dh_exact(a * (1 + d), f[:, k], feq[:, k])
        assert d < 1e-6 and lo < 0 < hi, (a, d, lo, hi)
    assert roots >= 2


def test_small_deviation_limit():
    """alpha - 2 against the first correction a3/(3 a2): the remainder falls like eps^2."""
    rems = []
    for eps in (4e-2, 2e-2, 1e-2):
        f, feq = _pair(6, 0.5, eps, seed=11)
        x = (feq - f) / f
        a2, a3 = (f * x ** 2).sum(axis=0), (f * x ** 3).sum(axis=0)
        alpha = O.entropic_alpha(f, feq)
        assert np.all(np.abs(alpha - 2) < 2 * eps)
        rems.append(np.abs(alpha - 2 - a3 / (3 * a2)).max())
    assert rems[0] / rems[1] > 3.0 and rems[1] / rems[2] > 3.0, rems


def test_equilibrium_gives_two():
    f, _, _ = O.entropic_equilibrium(np.array([1.0, 0.8]), np.array([[0.1, 0.0], [0.0, 0.2], [0.0, 0.0]]),
                                     np.full(2, T0))
    np.testing.assert_array_equal(O.entropic_alpha(f, f.copy()), [2.0, 2.0])


def test_no_root_inside_positivity_takes_alpha_max():
    """One population far above its equilibrium: the line reaches the positivity boundary
    before H climbs back to H[f]; alpha = alpha_max, where that population is zero."""
    rho, u, th = np.array([1.0]), np.zeros((3, 1)), np.array([T0])
    f, _, _ = O.entropic_equilibrium(rho, u, th)
    f[5, 0] *= 40.0
    r, uu, t = O.moments(f)
    feq, _, _ = O.entropic_equilibrium(r, uu, t)
    D = feq - f
    amax = (f[:, 0] / -D[:, 0])[D[:, 0] < 0].min()
    alpha = O.entropic_alpha(f, feq)
    assert alpha[0] == pytest.approx(amax, rel=1e-15)
    assert _dh_exact(amax, f[:, 0], feq[:, 0]) < 0


def test_h_theorem_and_conservation_over_steps():
    """Periodic 6x5x4 grid, random positive state, entropic equilibrium + entropic alpha,
    beta = 1/(2 tau + 1) with tau = 0.02 (alpha beta close to alpha): total H never grows and
    the conserved sums stay fixed."""
    rng = np.random.default_rng(3)
    shape = (2, 4, 5, 6)
    rho = 1 + 0.1 * rng.uniform(-1, 1, shape)
    th = T0 * (1 + 0.1 * rng.uniform(-1, 1, shape))
    u = 0.4 * CS * rng.uniform(-1, 1, (3,) + shape)
    f = O.init(rho, u, th, eq="entropic")
    f *= np.exp(0.05 * rng.uniform(-1, 1, f.shape))        # off equilibrium
    tot0 = O.totals(f)
    h_prev = O.boltzmann_h(np.moveaxis(f, 1, 0)).sum()
    for _ in range(6):
        f = O.step(f, 0.02, eq="entropic", collision="entropic")
        h = O.boltzmann_h(np.moveaxis(f, 1, 0)).sum()
        assert h <= h_prev + 1e-13 * abs(h_prev)
        h_prev = h
        np.testing.assert_allclose(O.totals(f), tot0, rtol=0, atol=1e-11 * np.abs(tot0).max())


def test_entropic_alpha_needs_entropic_equilibrium():
    f = O.init(np.ones((2, 1, 1, 2)), np.zeros((3, 2, 1, 1, 2)), np.full((2, 1, 1, 2), T0))
    with pytest.raises(ValueError):
        O.step(f, 0.1, eq="series", collision="entropic")
