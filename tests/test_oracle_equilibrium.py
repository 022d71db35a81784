"""Pins of the oracle's temperature weights and series equilibrium (App. B) against facts
fixed independently of the code:

* W~_i/(rho w_i) is the eta^4 Taylor polynomial of the Maxwellian ratio
  (1+eta)^(-3/2) exp(y eta / (2 (1+eta))), derived here with sympy;
* <W~, 1> = rho and <W~, c^2> = 3 rho theta hold exactly (traces imposed to c^10);
* R-bar has the closed form eta^4 (M6 - 13!!) / (5760 (1+eta)^2), M6 = <w, (c^2/theta0)^6>,
  which follows from the trace conditions; M6 is computed in exact rational arithmetic;
* the equilibrium reproduces rho, rho u and rho u^2 + 3 rho theta to round-off at any
  (u, theta), including Mach 2 (the conservation constraints of App. B);
* at theta = theta0 it reduces to the textbook third-order Hermite expansion of the
  Maxwellian, so its pressure tensor and third moment are the Maxwell-Boltzmann ones;
* it is equivariant under the cubic symmetry group.
"""

from fractions import Fraction
from itertools import permutations, product

import numpy as np
import pytest
import sympy as sp

from oracle import rd3q81 as O

LAT = O.velocity_set()
T0 = LAT.theta0
CS = np.sqrt(5.0 * T0 / 3.0)


def _series_coeffs():
    eta, y = sp.symbols("eta y")
    gen = (1 + eta) ** sp.Rational(-3, 2) * sp.exp(y * eta / (2 * (1 + eta)))
    ser = sp.series(gen, eta, 0, 5).removeO()
    return [sp.lambdify(y, sp.expand(ser).coeff(eta, k)) for k in range(5)]


def test_temperature_weights_match_maxwellian_series():
    coeffs = _series_coeffs()
    etas = np.array([-0.3, -0.1, 0.0, 0.05, 0.2, 0.3])
    W = O.temperature_weights(np.ones_like(etas), T0 * (1 + etas))      # [81, 6]
    y = LAT.c2 / T0
    for k, e in enumerate(etas):
        ref = np.array([sum(float(coeffs[m](yy)) * e ** m for m in range(5)) for yy in y])
        np.testing.assert_allclose(W[:, k] / LAT.w, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("eta", [-0.3, -0.15, 0.0, 0.1, 0.3])
def test_temperature_weight_traces(eta):
    rho = np.array([1.7])
    th = np.array([T0 * (1 + eta)])
    W = O.temperature_weights(rho, th)[:, 0]
    assert abs(W.sum() - rho[0]) < 1e-14
    assert abs(W @ LAT.c2 - 3 * rho[0] * th[0]) < 1e-13
    assert np.allclose(LAT.c.T @ W, 0.0, atol=1e-15)


def test_rbar_closed_form():
    t0 = Fraction(O.THETA0_TEXT)
    M6 = sum(w * (Fraction(int((h ** 2).sum()), 4) / t0) ** 6 for w, h in zip(LAT.w_exact, LAT.h))
    M6 = float(M6)
    etas = np.linspace(-0.3, 0.3, 13)
    rb = O.rbar(T0 * (1 + etas))
    ref = etas ** 4 * (M6 - 135135.0) / (5760.0 * (1 + etas) ** 2)
    np.testing.assert_allclose(rb, ref, rtol=1e-9, atol=1e-14)
    assert abs(M6 - 138243.35174) < 1e-4


def test_rbar_tensor_vanishes_at_theta0():
    rng = np.random.default_rng(3)
    u = rng.normal(size=(3, 7)) * 0.8
    R = O.rbar_tensor_contraction(np.full(7, T0), u)
    assert np.abs(R).max() < 1e-12


def _random_states(n, mach_max, eta_max, seed):
    rng = np.random.default_rng(seed)
    rho = 0.5 + rng.random(n)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    u = d * rng.random(n) * mach_max * CS
    th = T0 * (1 + eta_max * (2 * rng.random(n) - 1))
    return rho, u, th


@pytest.mark.parametrize("mach,eta", [(0.3, 0.05), (1.0, 0.2), (2.0, 0.3), (2.0, 0.0)])
def test_equilibrium_conserves(mach, eta):
    rho, u, th = _random_states(64, mach, eta, seed=int(mach * 10 + eta * 100))
    feq = O.equilibrium(rho, u, th)
    r, uu, t = O.moments(feq)
    np.testing.assert_allclose(r, rho, rtol=1e-13)
    np.testing.assert_allclose(uu, u, rtol=0, atol=1e-13 * (1 + np.abs(u).max()))
    np.testing.assert_allclose(t, th, rtol=1e-12)


def test_equilibrium_is_hermite_at_theta0():
    """At theta = theta0: Rb = 0, the R-bar tensor vanishes by 8th-order isotropy and
    W~ = rho w, leaving the third-order Hermite expansion of the Maxwellian."""
    rho, u, _ = _random_states(32, 1.0, 0.0, seed=11)
    th = np.full_like(rho, T0)
    feq = O.equilibrium(rho, u, th)
    xi = LAT.c @ u
    q = (u ** 2).sum(0)
    herm = LAT.w[:, None] * rho * (1 + xi / T0 + (xi ** 2 - T0 * q) / (2 * T0 ** 2)
                                   + (xi ** 3 - 3 * T0 * q * xi) / (6 * T0 ** 3))
    np.testing.assert_allclose(feq, herm, rtol=1e-12, atol=1e-15)


def test_pressure_tensor_and_third_moment_at_theta0():
    rho, u, _ = _random_states(16, 0.8, 0.0, seed=5)
    th = np.full_like(rho, T0)
    feq = O.equilibrium(rho, u, th)
    c = LAT.c
    P = np.einsum("ia,ib,in->abn", c, c, feq)
    Pref = rho * (T0 * np.eye(3)[:, :, None] + u[:, None, :] * u[None, :, :])
    np.testing.assert_allclose(P, Pref, rtol=0, atol=1e-12)
    Q = np.einsum("ia,ib,ic,in->abcn", c, c, c, feq)
    d = np.eye(3)
    Qref = rho * (np.einsum("an,bn,cn->abcn", u, u, u)
                  + T0 * (np.einsum("an,bc->abcn", u, d) + np.einsum("bn,ac->abcn", u, d)
                          + np.einsum("cn,ab->abcn", u, d)))
    np.testing.assert_allclose(Q, Qref, rtol=0, atol=1e-12)


def _cubic_group():
    mats = []
    for perm in permutations(range(3)):
        for signs in product((1, -1), repeat=3):
            M = np.zeros((3, 3))
            for r, (p, s) in enumerate(zip(perm, signs)):
                M[r, p] = s
            mats.append(M)
    return mats


def test_equilibrium_cubic_equivariance():
    rho, u, th = _random_states(8, 1.5, 0.25, seed=9)
    feq = O.equilibrium(rho, u, th)
    index = {tuple(h): i for i, h in enumerate(LAT.h)}
    group = _cubic_group()
    assert len(group) == 48
    for M in group:
        feq_r = O.equilibrium(rho, M @ u, th)
        # direction i of the rotated state equals direction sigma^-1(i) of the original
        perm = [index[tuple((M.T @ h).astype(int))] for h in LAT.h]
        np.testing.assert_allclose(feq_r, feq[perm], rtol=1e-12, atol=1e-14)
