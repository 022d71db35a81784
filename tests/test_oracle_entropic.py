"""Pins of the oracle's exact entropic equilibrium (Sec. III): the minimiser of
H = <f, log(f/w) - 1> under the conservation constraints, found by Newton on the paper's 5x5
moment system.  Checked against properties that define it rather than against its own code:

* the constraints: <f, {1, c, c^2}> = {rho, rho u, rho u^2 + 3 rho theta}, up to Mach 2;
* first-order optimality: log(f_i / w_i) lies in span{1, c_i, c_i^2} (least-squares residual
  at round-off), which is what "minimiser of H under these constraints" means;
* second-order: H strictly grows along every moment-preserving perturbation;
* positivity, and f = w rho at rest (u = 0, theta = theta0);
* the series equilibrium of App. B is its expansion: at theta0 the difference falls like u^4
  (the series is exact through u^3);
* cubic-symmetry equivariance.
"""

from itertools import permutations, product

import numpy as np
import pytest

from oracle import rd3q81 as O

LAT = O.velocity_set()
T0 = LAT.theta0
CS = np.sqrt(5.0 * T0 / 3.0)
PHI = np.concatenate([np.ones((81, 1)), LAT.c, LAT.c2[:, None]], axis=1)


def _states(n, mach, eta, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    u = d * mach * CS * rng.uniform(0.5, 1.0, n)
    rho = rng.uniform(0.5, 1.5, n)
    th = T0 * (1 + eta * rng.uniform(-1, 1, n))
    return rho, u, th


@pytest.mark.parametrize("mach,eta", [(0.0, 0.0), (0.5, 0.1), (1.0, 0.3), (1.5, 0.2), (2.0, 0.3)])
def test_constraints_and_positivity(mach, eta):
    rho, u, th = _states(48, mach, eta, seed=int(10 * mach + 100 * eta))
    f, lam, it = O.entropic_equilibrium(rho, u, th)
    assert not np.isnan(f).any() and it < 40
    assert np.all(f > 0)
    r, uu, t = O.moments(f)
    np.testing.assert_allclose(r, rho, rtol=1e-13)
    np.testing.assert_allclose(uu, u, rtol=0, atol=1e-13 * (1 + np.abs(u).max()))
    np.testing.assert_allclose(t, th, rtol=1e-12)


def test_rest_state_is_weights():
    rho = np.array([0.7, 1.0, 1.9])
    f, lam, _ = O.entropic_equilibrium(rho, np.zeros((3, 3)), np.full(3, T0))
    np.testing.assert_allclose(f, LAT.w[:, None] * rho, rtol=1e-14)
    assert np.abs(lam).max() < 1e-14


@pytest.mark.parametrize("mach,eta", [(0.5, 0.1), (2.0, 0.3)])
def test_first_order_optimality(mach, eta):
    """log(f/w) must be an affine function of (1, c, c^2): the Lagrange condition of
    minimising H under the five linear constraints."""
    rho, u, th = _states(16, mach, eta, seed=3)
    f, _, _ = O.entropic_equilibrium(rho, u, th)
    g = np.log(f / LAT.w[:, None])
    coef, *_ = np.linalg.lstsq(PHI, g, rcond=None)
    resid = g - PHI @ coef
    assert np.abs(resid).max() < 1e-10 * (1 + np.abs(g).max())


@pytest.mark.parametrize("mach,eta", [(0.5, 0.1), (1.5, 0.2)])
def test_h_grows_along_moment_preserving_perturbations(mach, eta):
    rho, u, th = _states(6, mach, eta, seed=5)
    f, _, _ = O.entropic_equilibrium(rho, u, th)
    rng = np.random.default_rng(7)
    for k in range(f.shape[1]):
        fk = f[:, k]
        h0 = O.boltzmann_h(fk)
        # relative perturbations d_i = f_i v_i with sum_i f_i v_i phi_i = 0: v spans the
        # 76-dimensional null space of the f-weighted constraint matrix
        q, _ = np.linalg.qr(np.concatenate([PHI * fk[:, None], np.eye(81)], axis=1))
        null = q[:, 5:81]
        for _ in range(20):
            v = null @ rng.normal(size=76)
            v *= 1e-3 / np.abs(v).max()
            d = fk * v
            assert np.abs(PHI.T @ d).max() < 1e-13 * fk.sum()
            assert O.boltzmann_h(fk + d) > h0
            assert O.boltzmann_h(fk - d) > h0


def test_series_equilibrium_is_its_expansion():
    """At theta0 the series form is exact through u^3, so the two differ at O(u^4)."""
    rng = np.random.default_rng(11)
    d = rng.normal(size=(3, 8))
    d /= np.linalg.norm(d, axis=0)
    rho = np.ones(8)
    th = np.full(8, T0)
    errs = []
    for mach in (0.2, 0.1, 0.05):
        u = d * mach * CS
        fe, _, _ = O.entropic_equilibrium(rho, u, th)
        fs = O.equilibrium(rho, u, th)
        errs.append(np.abs(fe - fs).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12.0 < r1 < 20.0 and 14.0 < r2 < 18.0, errs


def test_cubic_equivariance():
    rho, u, th = _states(5, 1.2, 0.2, seed=13)
    f, _, _ = O.entropic_equilibrium(rho, u, th)
    index = {tuple(h): i for i, h in enumerate(LAT.h)}
    for perm in list(permutations(range(3)))[::2]:
        for signs in list(product((1, -1), repeat=3))[::3]:
            M = np.zeros((3, 3))
            for r, (p, s) in enumerate(zip(perm, signs)):
                M[r, p] = s
            fr, _, _ = O.entropic_equilibrium(rho, M @ u, th)
            pi = [index[tuple((M.T @ h).astype(int))] for h in LAT.h]
            np.testing.assert_allclose(fr, f[pi], rtol=1e-12, atol=1e-16)
