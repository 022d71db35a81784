"""Pins of the oracle's exact temperature-dependent weights W(theta) (App. B, Eq. (zeroveleq):
W_i = w_i A G^(4 c_i^2), G the root of theta'(G) = F2 / (3 theta0 F0)) and of the series
equilibrium that uses them.  Checked against what fixes them, not their own formulas:

* the two conditions that define them: <W, 1> = 1, <W, c^2> = 3 theta (and <W, c> = 0);
* the exact entropic equilibrium at rest: rho W(theta) = f_eq(rho, u = 0, theta), which the
  5x5 multiplier Newton finds independently;
* the eta^4 series W~ of Eq. (zeroveleqseries) is W's expansion: the difference falls like eta^5;
* theta = theta0 gives the weights themselves; theta'(G) rises monotonically (Fig. "theta_G");
* the series equilibrium with exact weights equals rho W at u = 0 and keeps mass, momentum and
  energy exactly, like the one with W~ (energy only if Rb comes from the same weights).
"""

import numpy as np
import pytest

from oracle import rd3q81 as O

LAT = O.velocity_set()
T0 = LAT.theta0
CS = np.sqrt(5.0 * T0 / 3.0)


def test_defining_moments():
    th = T0 * np.array([0.25, 0.4, 0.6, 0.9, 1.0, 1.3, 2.0, 3.5])
    W = O.temperature_weights_exact(np.ones(th.size), th)
    np.testing.assert_allclose(W.sum(axis=0), 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(LAT.c.T @ W, 0.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(LAT.c2 @ W, 3.0 * th, rtol=1e-14)
    assert np.all(W > 0)


def test_equals_entropic_equilibrium_at_rest():
    rng = np.random.default_rng(4)
    th = T0 * rng.uniform(0.3, 2.5, 12)
    rho = rng.uniform(0.5, 2.0, 12)
    W = O.temperature_weights_exact(rho, th)
    fe, _, _ = O.entropic_equilibrium(rho, np.zeros((3, 12)), th)
    np.testing.assert_allclose(W, fe, rtol=1e-12, atol=0)


def test_series_is_its_expansion():
    errs = []
    for eta in (0.04, 0.02, 0.01):
        th = T0 * np.array([1 + eta, 1 - eta])
        errs.append(np.abs(O.temperature_weights_exact(np.ones(2), th) - O.temperature_weights(np.ones(2), th)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 26.0 < r1 < 38.0 and 26.0 < r2 < 38.0, errs          # 2^5 = 32


def test_reference_temperature_and_monotone_map():
    np.testing.assert_allclose(O.temperature_weights_exact(np.ones(1), np.array([T0]))[:, 0], LAT.w, rtol=1e-14)
    # theta'(G): at higher theta every moving shell gains weight relative to the rest particle
    th = T0 * np.linspace(0.3, 3.0, 40)
    W = O.temperature_weights_exact(np.ones(th.size), th)
    G4 = W[1] / (W[0] * LAT.w[1] / LAT.w[0])                 # G^4 from an SC-1 direction (c^2 = 1)
    assert np.all(np.diff(G4) > 0)


@pytest.mark.parametrize("mach", [0.0, 0.5, 1.0])
def test_series_equilibrium_with_exact_weights(mach):
    rng = np.random.default_rng(8)
    n = 16
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    u = d * mach * CS
    rho = rng.uniform(0.5, 1.5, n)
    th = T0 * rng.uniform(0.5, 1.8, n)
    f = O.equilibrium(rho, u, th, weights="exact")
    r, uu, t = O.moments(f)
    np.testing.assert_allclose(r, rho, rtol=1e-13)
    np.testing.assert_allclose(uu, u, rtol=0, atol=1e-13)
    # energy: exact only when Rb and its tensor are taken from the same weights as W
    np.testing.assert_allclose(t, th, rtol=1e-12)
    if mach == 0.0:
        np.testing.assert_allclose(f, O.temperature_weights_exact(rho, th), rtol=1e-13)
    # and it reduces to the standard series equilibrium at theta0
    f0 = O.equilibrium(rho, u, np.full(n, T0), weights="exact")
    np.testing.assert_allclose(f0, O.equilibrium(rho, u, np.full(n, T0)), rtol=1e-12, atol=1e-16)
