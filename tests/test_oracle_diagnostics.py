"""Pins of the oracle's kinetic energy and enstrophy (Sec. IV C) against closed forms.

For u = U0 (sin X cos Y cos Z, -cos X sin Y cos Z, 0), X = 2 pi x / N (any grid offset), rho = 1,
the grid means of sin^2 and cos^2 over whole periods are 1/2, so KE = U0^2 / 8; second-order
central differences turn d/dx of sin X into cos X sin(2 pi / N), so the discrete vorticity has
w^2 mean (3/4) U0^2 sin^2(2 pi / N) and eps = (3/8) U0^2 sin^2(2 pi / N).  A uniform flow has
zero enstrophy; rho scales both linearly; the shear u_y = Om x has w_z = Om everywhere
(central and one-sided second-order differences are exact on linear fields), on a grid with
non-periodic x."""

import numpy as np
import pytest

from oracle import rd3q81 as O

LAT = O.velocity_set()
T0 = LAT.theta0


def _state(u, rho=None):
    S = u.shape[1:]
    rho = np.ones(S) if rho is None else rho
    return O.init(rho, u, np.full(S, T0))


def _tgv(N, U0, nz=None):
    nz = nz or N
    s = np.arange(2)[:, None, None, None] * 0.5
    z, y, x = np.meshgrid(np.arange(nz), np.arange(N), np.arange(N), indexing="ij")
    X, Y, Z = (2 * np.pi * (x + s) / N, 2 * np.pi * (y + s) / N, 2 * np.pi * (z + s) / nz)
    return np.stack([U0 * np.sin(X) * np.cos(Y) * np.cos(Z), -U0 * np.cos(X) * np.sin(Y) * np.cos(Z),
                     np.zeros_like(X)])


@pytest.mark.parametrize("N", [8, 12])
def test_tgv_closed_forms(N):
    U0 = 0.1
    f = _state(_tgv(N, U0))
    ke, ens = O.diagnostics(f)
    assert ke == pytest.approx(U0 ** 2 / 8, rel=1e-12)
    assert ens == pytest.approx(3 / 8 * U0 ** 2 * np.sin(2 * np.pi / N) ** 2, rel=1e-12)
    # rho scales both
    f2 = O.init(np.full((2, N, N, N), 1.3), _tgv(N, U0), np.full((2, N, N, N), T0))
    ke2, ens2 = O.diagnostics(f2)
    assert ke2 == pytest.approx(1.3 * ke, rel=1e-12) and ens2 == pytest.approx(1.3 * ens, rel=1e-12)


def test_uniform_flow_and_linear_shear():
    u = np.zeros((3, 2, 4, 6, 5))
    u[0] = 0.05
    ke, ens = O.diagnostics(_state(u))
    assert ke == pytest.approx(0.5 * 0.05 ** 2, rel=1e-12) and abs(ens) < 1e-28
    # shear linear in x (x non-periodic: one-sided end differences), uniform in y and z
    Om = 1e-3
    z, y, x = np.meshgrid(np.arange(4), np.arange(6), np.arange(9), indexing="ij")
    s = np.arange(2)[:, None, None, None] * 0.5
    u = np.zeros((3, 2, 4, 6, 9))
    u[1] = Om * (x + s)                                  # u_y = Om x: w_z = Om everywhere
    ke, ens = O.diagnostics(_state(u), x_periodic=False)
    assert ens == pytest.approx(0.5 * Om ** 2, rel=1e-10)


@pytest.mark.parametrize("comp", [0, 1, 2])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_single_mode_shear_waves(comp, axis):
    """u_comp = A sin(2 pi q / N_axis) along one axis of a 9 x 7 x 5 grid: the curl is the
    derivative along that axis, A cos(.) sin(2 pi / N_axis), unless axis = comp (no curl);
    eps = A^2 sin^2(2 pi / N_axis) / 4.  Distinct N per axis catch a swapped derivative."""
    A = 0.02
    dims = (5, 7, 9)                     # z, y, x
    z, y, x = np.meshgrid(*(np.arange(n) for n in dims), indexing="ij")
    s = np.arange(2)[:, None, None, None] * 0.5
    q = (x, y, z)[axis] + s
    n_ax = (dims[2], dims[1], dims[0])[axis]
    u = np.zeros((3, 2) + dims)
    u[comp] = A * np.sin(2 * np.pi * q / n_ax)
    ke, ens = O.diagnostics(_state(u))
    assert ke == pytest.approx(A ** 2 / 4, rel=1e-12)
    ref = 0.0 if axis == comp else A ** 2 * np.sin(2 * np.pi / n_ax) ** 2 / 4
    assert ens == pytest.approx(ref, rel=1e-12, abs=1e-30)
