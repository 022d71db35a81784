"""Pins of the oracle's bounce-back wall (the Sod setup of Sec. IV A: "standard bounce back" on the
x faces; the paper gives no formula, the reading is stated in ``oracle.rd3q81.stream``).  Checked
against what fixes it, not against its own code:

* brute force: every single population of a small grid is streamed on its own and must land
  where a push-form mover puts it -- translated by c_i between physical positions (P sites at n,
  R sites at n + 1/2), or, if that position's x index lies outside the fluid, back on its own
  site with the reversed velocity;
* time reversal: streaming, reversing every velocity, streaming again gives the reversed start;
* streaming only permutes the values; a closed box (walls on both x faces) keeps mass and energy
  to rounding through full steps, and the rest state is a fixed point.
"""

import numpy as np
import pytest

from oracle import rd3q81 as O

LAT = O.velocity_set()
T0 = LAT.theta0
OPP = np.array([int(np.flatnonzero(np.all(LAT.h == -LAT.h[i], axis=1))[0]) for i in range(LAT.q)])
BB = ("bounce_back", "bounce_back")


def _push_target(s, i, n, shape, faces):
    """Where a unit population at sublattice s, direction i, index n = (x, y, z) goes in one
    step, computed from physical positions: (sublattice, direction, index)."""
    nz, ny, nx = shape
    pos2 = 2 * np.array(n) + s + LAT.h[i]          # twice the arrival position
    if np.all(pos2 % 2 == 0):
        t_sub, idx = 0, pos2 // 2
    else:
        assert np.all(pos2 % 2 == 1)
        t_sub, idx = 1, (pos2 - 1) // 2
    x = int(idx[0])
    if (x < 0 and faces[0] == "bounce_back") or (x >= nx and faces[1] == "bounce_back"):
        return s, int(OPP[i]), tuple(n)
    return t_sub, i, (x, int(idx[1]) % ny, int(idx[2]) % nz)    # x may lie beyond an open face


@pytest.mark.parametrize("faces", [BB, ("zero_gradient", "bounce_back"), ("bounce_back", "eq_inflow")])
def test_single_populations_brute_force(faces):
    nz, ny, nx = 2, 3, 9
    shape = (nz, ny, nx)
    rng = np.random.default_rng(1)
    zero_in = (np.zeros(LAT.q), np.zeros(LAT.q))        # inflow ghosts hold 0: no extra values
    checked = 0
    for s in (0, 1):
        for i in range(LAT.q):
            for x in range(nx):
                if faces[0] == "zero_gradient" and x == 0:
                    continue                        # copied into the open face's ghosts
                n = (x, int(rng.integers(ny)), int(rng.integers(nz)))
                f = np.zeros((2, LAT.q) + shape)
                f[s, i, n[2], n[1], n[0]] = 1.0
                g = O.stream(f, faces, zero_in)
                t_sub, t_i, (tx, ty, tz) = _push_target(s, i, n, shape, faces)
                if not 0 <= tx < nx:
                    assert np.count_nonzero(g) == 0   # left through the open face
                    continue
                assert g[t_sub, t_i, tz, ty, tx] == 1.0, (s, i, n)
                assert np.count_nonzero(g) == 1, (s, i, n)
                checked += 1
    assert checked > 2 * LAT.q * (nx - 2)


def test_time_reversal():
    rng = np.random.default_rng(2)
    f = rng.uniform(0.5, 1.5, (2, LAT.q, 3, 4, 11))
    g = O.stream(f, BB)
    back = O.stream(g[:, OPP], BB)
    np.testing.assert_array_equal(back, f[:, OPP])


def test_streaming_permutes_values():
    rng = np.random.default_rng(3)
    f = rng.uniform(0.5, 1.5, (2, LAT.q, 2, 3, 7))
    g = O.stream(f, BB)
    np.testing.assert_array_equal(np.sort(g.ravel()), np.sort(f.ravel()))


def test_closed_box_conserves_mass_and_energy():
    rng = np.random.default_rng(4)
    shape = (2, 3, 4, 12)
    rho = 1 + 0.05 * rng.uniform(-1, 1, shape)
    th = T0 * (1 + 0.05 * rng.uniform(-1, 1, shape))
    u = 0.3 * np.sqrt(5 * T0 / 3) * rng.uniform(-1, 1, (3,) + shape)
    f = O.init(rho, u, th)
    t0 = O.totals(f)
    bc = (("bounce_back",), ("bounce_back",))
    for _ in range(5):
        f = O.step(f, 0.2, bc)
        t = O.totals(f)
        assert abs(t[0] - t0[0]) <= 1e-13 * abs(t0[0])
        assert abs(t[4] - t0[4]) <= 1e-13 * abs(t0[4])


def test_rest_state_is_fixed_point():
    shape = (2, 2, 3, 10)
    f = O.init(np.ones(shape), np.zeros((3,) + shape), np.full(shape, T0))
    g = O.run(f, 0.3, 3, (("bounce_back",), ("bounce_back",)))
    np.testing.assert_allclose(g, f, rtol=0, atol=1e-15)
