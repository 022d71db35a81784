"""FP64 CPU oracle for one RD3Q81 lattice Boltzmann step.

Paper: M. Atif, N. H. Maruthi, P. K. Kolluru, C. Thantanapally, S. Ansumali,
"Lattice Boltzmann Model for Transonic Flows" (arXiv 2409.05114).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import this module.  The product path (the CUDA library
and its Python binding) never imports it, and the two share no code, constant table or
helper: this file rebuilds the velocity set from the paper's table on its own.

Everything is plain numpy float64, in the paper's order and notation, so that it can be
read against the paper line by line:

* ``velocity_set``        Sec. III + Table "tab:weights": the ten RD3Q81 shells, their
                          weights as quintic polynomials of theta0, w_0 = 1 - sum(others).
* ``moments``             Sec. II, Eq. (conslaws): rho, rho*u, rho*u^2 + 3*rho*theta.
* ``temperature_weights`` App. B, Eq. (zeroveleqseries): the eta^4 series W~_i(theta).
* ``temperature_weights_exact`` App. B, Eq. (zeroveleq): W_i = w_i A G^(4 c_i^2) with G the root of
                          theta'(G) = F2/(3 theta0 F0), Eq. (f0f2geqn).
* ``equilibrium``         App. B, "Discrete equilibrium at nonzero velocity": f~eq with
                          f^(2), f^(3), R-bar and the tensor R-bar_{kappa alpha zeta eta},
                          the last two as explicit 81-term sums over W~/rho.
* ``entropic_equilibrium`` Sec. III: the exact minimiser of H = <f, log(f/w) - 1>, i.e.
                          w rho exp(mu + zeta.c + gamma c^2), by Newton on the paper's 5x5
                          moment system; ``boltzmann_h`` is H itself.
* ``stream``              Sec. II, Eq. (discretelbm), left side: f_i moves by c_i in one
                          step.  Half-integer links join the primary lattice (P, integer
                          positions) and the replica lattice (R, positions + (1/2,1/2,1/2)),
                          Sec. I (replica grid) and Sec. V (body-centred cubic lattice).
* ``collide``             Sec. II, Eq. (discretelbm), right side: alpha = 2 (BGK) or the
                          entropic alpha, beta = dt / (2 tau + dt) with dt = 1.
* ``entropic_alpha``      Sec. II, Eq. (delH): the nontrivial root of
                          H[f + alpha (feq - f)] - H[f] = 0 (``entropic_delta_h``).
* ``diagnostics``         Sec. IV C: mean kinetic energy and mean enstrophy (curl by central
                          differences on each sublattice).
* ``fill_ghosts_x``       Boundary layers in x.  The paper names its own boundary
                          conditions without formulas; this oracle implements the four the
                          library offers (periodic, zero-gradient outflow, equilibrium
                          inflow, and the bounce-back wall of the Sod setup in Sec. IV A,
                          applied in ``stream``), each defined in its docstring.

Parity pins (tests/test_oracle_*.py): lattice identities in exact arithmetic, the paper's
printed moment-error column, W~ against its closed-form generating function, equilibrium
moments, uniform-state fixed points, conservation on periodic grids, cubic-symmetry
equivariance, the closed-form sound speed, the shear-wave viscosity nu = tau theta0 that fixes the
relaxation rate beta of ``collide`` (Sec. II) and the exact Sod/Riemann solution; the entropic
equilibrium's constraints, optimality conditions and small-velocity limit; Delta H against the
definition of H in 50-digit arithmetic, the root's small-deviation limit alpha -> 2 + a3/(3 a2)
and the discrete H theorem of whole steps; the exact W(theta) against the entropic equilibrium at
rest and its eta^4 series.  No function here is "parity unpinned".

Array conventions (all float64):
    populations  f[s, i, z, y, x]   s = 0 (P) or 1 (R), i = direction (this module's order)
    fields       rho[s, z, y, x], theta[s, z, y, x], u[a, s, z, y, x] with a = x, y, z
"""

from __future__ import annotations

from fractions import Fraction
from itertools import permutations, product

import numpy as np

# theta0 as printed under Table "tab:weights" (Sec. III).
THETA0_TEXT = "0.821035006329447750282591763"
THETA0 = float(THETA0_TEXT)

# Table "tab:weights": shell name, one generating velocity in half units h = 2c, and the
# weight as {power of theta0: integer coefficient} over an integer denominator.
_SHELLS = (
    ("SC-1", (2, 0, 0), {1: 388800, 2: -2508408, 3: 7033852, 4: -7856469, 5: 2838528}, 486000),
    ("SC-2", (4, 0, 0), {1: -388800, 2: 3091608, 3: -8269102, 4: 8694819, 5: -2838528}, 3888000),
    ("SC-3", (6, 0, 0), {1: 388800, 2: -3199608, 3: 8977852, 4: -9120069, 5: 2838528}, 30618000),
    ("SC-4", (8, 0, 0), {1: -97200, 2: 809352, 3: -2315338, 4: 2396961, 5: -709632}, 108864000),
    ("FCC-1", (2, 2, 0), {3: 8, 4: -9}, 12),
    ("FCC-2", (4, 4, 0), {3: -2, 4: 9}, 768),
    ("BCC-1/2", (1, 1, 1), {2: 24300, 3: -103834, 4: 126963, 5: -44352}, 7776),
    ("BCC-1", (2, 2, 2), {2: -24300, 3: 189022, 4: -328275, 5: 177408}, 272160),
    ("BCC-3/2", (3, 3, 3), {2: 2700, 3: -24778, 4: 67995, 5: -44352}, 699840),
    ("BCC-5/2", (5, 5, 5), {2: -972, 3: 11818, 4: -43371, 5: 44352}, 68040000),
)


def shell_weight_exact(coeffs: dict, den: int, theta0: Fraction) -> Fraction:
    """One row of Table "tab:weights": sum_k coeffs[k] * theta0**k / den, exactly."""
    return sum((Fraction(c) * theta0 ** k for k, c in coeffs.items()), Fraction(0)) / den


def _shell_vectors(gen):
    """All distinct vectors obtained from ``gen`` by permuting and sign-flipping components
    (the SC, FCC and BCC shells of App. A)."""
    out = set()
    for perm in permutations(gen):
        for signs in product((1, -1), repeat=3):
            out.add(tuple(s * p for s, p in zip(signs, perm)))
    return sorted(out)


class Lattice:
    """The RD3Q81 velocity set (Sec. III, Table "tab:weights").

    Attributes
    ----------
    h      : int64[81, 3]  velocities in half units, h = 2 c
    c      : float64[81, 3] velocities c_i (components in {0, +-1/2, +-1, ..., +-4})
    c2     : float64[81]   |c_i|^2
    w      : float64[81]   weights w_i = W_i(theta0); w_0 = 1 - sum of the others
    shell  : list[str]     shell name of each direction ("rest" for i = 0)
    theta0 : float         reference temperature
    """

    def __init__(self, theta0_text: str = THETA0_TEXT):
        t0 = Fraction(theta0_text)
        hs, ws, names = [(0, 0, 0)], [None], ["rest"]
        for name, gen, coeffs, den in _SHELLS:
            wt = shell_weight_exact(coeffs, den, t0)
            for v in _shell_vectors(gen):
                hs.append(v)
                ws.append(wt)
                names.append(name)
        ws[0] = Fraction(1) - sum(ws[1:], Fraction(0))
        self.h = np.array(hs, dtype=np.int64)
        self.c = self.h.astype(np.float64) / 2.0
        self.c2 = (self.c ** 2).sum(axis=1)
        self.w = np.array([float(x) for x in ws])
        self.w_exact = ws
        self.shell = names
        self.theta0 = float(t0)
        self.q = len(hs)


_LAT = None


def velocity_set() -> Lattice:
    """The (cached) RD3Q81 lattice."""
    global _LAT
    if _LAT is None:
        _LAT = Lattice()
    return _LAT


# ---------------------------------------------------------------------------------------
# Moments, Sec. II Eq. (conslaws)
# ---------------------------------------------------------------------------------------

def moments(f: np.ndarray, lat: Lattice | None = None):
    """rho = <f, 1>, rho u_a = <f, c_a>, rho u^2 + 3 rho theta = <f, c^2>.

    ``f`` has the direction index first: f[i, ...].  Returns (rho, u[3, ...], theta).
    """
    lat = lat or velocity_set()
    rho = np.tensordot(np.ones(lat.q), f, axes=(0, 0))
    j = np.tensordot(lat.c.T, f, axes=(1, 0))
    e = np.tensordot(lat.c2, f, axes=(0, 0))
    u = j / rho
    theta = (e - rho * (u ** 2).sum(axis=0)) / (3.0 * rho)
    return rho, u, theta


# ---------------------------------------------------------------------------------------
# Equilibrium, App. B
# ---------------------------------------------------------------------------------------

def temperature_weights(rho: np.ndarray, theta: np.ndarray, lat: Lattice | None = None):
    """W~_i(theta), App. B Eq. (zeroveleqseries), kept to eta^4 as printed there.

    W~_i = rho w_i [1 + eta/2 (y-3) + eta^2/8 (y^2 - 10y + 15)
                    + eta^3/48 (y^3 - 21y^2 + 105y - 105)
                    + eta^4/384 (y^4 - 36y^3 + 378y^2 - 1260y + 945)],
    with y_i = c_i^2 / theta0 and eta = theta/theta0 - 1.   Returns W[i, ...].
    """
    lat = lat or velocity_set()
    t0 = lat.theta0
    eta = theta / t0 - 1.0
    shape = (lat.q,) + (1,) * np.ndim(theta)
    y = (lat.c2 / t0).reshape(shape)
    w = lat.w.reshape(shape)
    # the bracket's coefficient of eta^k, per direction
    p1 = (y - 3.0) / 2.0
    p2 = (y ** 2 - 10.0 * y + 15.0) / 8.0
    p3 = (y ** 3 - 21.0 * y ** 2 + 105.0 * y - 105.0) / 48.0
    p4 = (y ** 4 - 36.0 * y ** 3 + 378.0 * y ** 2 - 1260.0 * y + 945.0) / 384.0
    poly = 1.0 + eta * p1 + eta ** 2 * p2 + eta ** 3 * p3 + eta ** 4 * p4
    return rho * w * poly


def temperature_weights_exact(rho: np.ndarray, theta: np.ndarray, lat: Lattice | None = None,
                              tol: float = 1e-12, max_iter: int = 100):
    """Exact temperature-dependent weights of App. B, Eq. (zeroveleq):

        W_i(theta) = w_i A G^(4 c_i^2),   A = 1 / F0(G),   theta' = theta/theta0 = F2(G) / (3 theta0 F0(G)),

    F0(G) = <w, G^(4 c^2)>, F2(G) = <w, c^2 G^(4 c^2)> (Eq. (f0f2geqn)), i.e. the weights that
    keep mass <W, 1> = 1 and energy <W, c^2> = 3 theta.  The paper solves the 1-D relation
    theta'(G) for G "with any iterative solver"; here in the variable g = 4 ln G, so that
    G^(4 c^2) = exp(g c^2) (no large powers): Newton on r(g) = F2/F0 - 3 theta, whose slope
    <c^4> - <c^2>^2 under the normalised weights is positive (a variance), from the paper's
    series multiplier g0 = 1/(2 theta0) - 1/(2 theta) (the sum of its gamma^(0) series), until a
    step is below tol (1 + |g|).  Returns rho * W [81, ...]; NaN where it did not converge."""
    lat = lat or velocity_set()
    rho = np.asarray(rho, dtype=np.float64)
    th = np.asarray(theta, dtype=np.float64)
    S = th.shape
    t1 = th.reshape(-1)
    g = 0.5 / lat.theta0 - 0.5 / t1
    w, c2 = lat.w[:, None], lat.c2[:, None]
    done = np.zeros(t1.size, dtype=bool)
    for _ in range(max_iter):
        e = w * np.exp(g * c2)
        F0, F2, F4 = e.sum(axis=0), (e * c2).sum(axis=0), (e * c2 * c2).sum(axis=0)
        step = (F2 / F0 - 3.0 * t1) / (F4 / F0 - (F2 / F0) ** 2)
        g = np.where(done, g, g - step)
        done |= np.abs(step) <= tol * (1.0 + np.abs(g))      # quadratic: the error left is ~step^2
        if done.all():
            break
    W = w * np.exp(g * c2) / (w * np.exp(g * c2)).sum(axis=0)
    W[:, ~done] = np.nan
    return (rho.reshape(-1) * W).reshape((lat.q,) + S) if rho.ndim else rho * W.reshape((lat.q,) + S)


def rbar(theta: np.ndarray, lat: Lattice | None = None, Wn: np.ndarray | None = None) -> np.ndarray:
    """Rb = <W~/rho, c^4> / (15 theta^2) - 1 (App. B), as an explicit 81-term sum.
    ``Wn`` may pass W~/rho at these temperatures if the caller already has it."""
    lat = lat or velocity_set()
    th = np.asarray(theta, dtype=np.float64).reshape(-1)
    if Wn is None:
        Wn = temperature_weights(np.ones_like(th), th, lat)
    return (lat.c2 ** 2) @ Wn / (15.0 * th ** 2) - 1.0


def rbar_tensor_contraction(theta: np.ndarray, u: np.ndarray, lat: Lattice | None = None,
                            Wn: np.ndarray | None = None):
    """u_a u_z u_e c_ix Rb_{x a z e} for every direction i (App. B), with
    Rb_{k a z e} = <W~/rho, c_k c_a c_z c_e> / theta^2 - Delta_{a k e z} written out as
    sum_j (W~_j/rho)(c_j.c_i)(c_j.u)^3 / theta^2 - 3 u^2 (u.c_i).   Returns [81, n].
    ``Wn`` may pass W~/rho at these temperatures if the caller already has it."""
    lat = lat or velocity_set()
    th = np.asarray(theta, dtype=np.float64).reshape(-1)
    u1 = np.asarray(u, dtype=np.float64).reshape(3, -1)
    if Wn is None:
        Wn = temperature_weights(np.ones_like(th), th, lat)
    xi = lat.c @ u1
    q = (u1 ** 2).sum(axis=0)
    G = lat.c @ lat.c.T                                   # c_i . c_j   [81, 81]
    return G @ (Wn * xi * xi * xi) / th ** 2 - 3.0 * q * xi


def equilibrium(rho: np.ndarray, u: np.ndarray, theta: np.ndarray, lat: Lattice | None = None,
                weights: str = "series"):
    """Series entropic equilibrium f~eq_i(rho, u, theta) of App. B (nonzero velocity):

        f~eq_i = W~_i(theta) [1 + u.c_i/theta + f_i^(2) + f_i^(3)]

        f^(2) = u_a u_b (c_a c_b - theta delta_ab) / (2 theta^2)
                - (5/3) u^2/(2 theta^2) * Rb/(2 + 5 Rb) * (c^2 - 3 theta)
        f^(3) = u_a u_b u_g (c_a c_b c_g - theta c_k Delta_abgk) / (6 theta^3)
                - [5/(6 theta^3) * Rb u^2/(2 + 5 Rb)] (u.c) (c^2 - 3 theta)
                + (5 (u.c) u^2 Rb - u_a u_z u_e c_x Rb_{x a z e}) / (6 theta^2)

    with  Rb_{k a z e} = <W~/rho, c_k c_a c_z c_e> / theta^2 - Delta_{a k e z}
    and   Rb           = <W~/rho, c^4> / (15 theta^2) - 1.

    W~ in the two Rb definitions is taken per unit density (W~/rho), which is the reading
    that makes both vanish at theta = theta0.  The contractions are written out:
        u_a u_b u_g c_k Delta_abgk         = 3 u^2 (u.c)
        u_a u_z u_e c_ix Rb_{x a z e}      = sum_j (W~_j/rho) (c_j.c_i) (c_j.u)^3 / theta^2
                                             - 3 u^2 (u.c_i)
    ``weights`` = "exact" takes the exact W(theta) of Eq. (zeroveleq) in place of the eta^4
    series W~ (in W~ itself and in both Rb).
    Inputs are arrays over sites (any shape S, u is [3, *S]); returns feq[81, *S].
    """
    lat = lat or velocity_set()
    rho = np.asarray(rho, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    S = rho.shape
    rho1, th = rho.reshape(-1), theta.reshape(-1)
    u1 = u.reshape(3, -1)

    if weights == "series":
        W = temperature_weights(rho1, th, lat)           # [81, n]
    elif weights == "exact":
        W = temperature_weights_exact(rho1, th, lat)
    else:
        raise ValueError(weights)
    q = (u1 ** 2).sum(axis=0)                             # u^2
    xi = lat.c @ u1                                       # u.c_i      [81, n]
    c2 = lat.c2[:, None]
    Wn = W / rho1                                         # W~ / rho
    Rb = rbar(th, lat, Wn)
    Rcontr = rbar_tensor_contraction(th, u1, lat, Wn)

    K = Rb / (2.0 + 5.0 * Rb)
    f1 = xi / th
    f2 = ((xi ** 2 - th * q) / (2.0 * th ** 2)
          - (5.0 / 3.0) * q / (2.0 * th ** 2) * K * (c2 - 3.0 * th))
    f3 = ((xi * xi * xi - th * 3.0 * q * xi) / (6.0 * th ** 3)
          - (5.0 / (6.0 * th ** 3) * K * q) * xi * (c2 - 3.0 * th)
          + (5.0 * xi * q * Rb - Rcontr) / (6.0 * th ** 2))
    feq = W * (1.0 + f1 + f2 + f3)
    return feq.reshape((lat.q,) + S)


def entropic_equilibrium(rho, u, theta, lat: Lattice | None = None, tol: float = 1e-12,
                         max_iter: int = 100):
    """Exact discrete entropic equilibrium of Sec. III:

        f_i = w_i rho exp(mu + zeta . c_i + gamma c_i^2),

    the minimiser of H = <f, log(f/w) - 1> under <f, {1, c, c^2}> = {rho, rho u,
    rho u^2 + 3 rho theta}.  The multipliers are found as the paper describes: with a guess
    f~ = w rho exp(mu0 + zeta0.c + gamma0 c^2), linearise exp(x) ~ 1 + x in the correction
    (mu^, zeta^, gamma^), solve the 5x5 system whose matrix is <f~, phi_a phi_b> and whose
    right side is (target moments - <f~, phi_a>), phi = (1, c_x, c_y, c_z, c^2), add the
    correction and repeat (Newton's method on the multipliers).  The first guess is the
    continuous Maxwellian's multipliers relative to w ~ exp(-c^2/(2 theta0)):
    mu0 = -(3/2) ln(theta/theta0) - u^2/(2 theta), zeta0 = u/theta,
    gamma0 = 1/(2 theta0) - 1/(2 theta).

    Safeguard (not in the paper, inactive whenever the full step works): the correction is
    the Newton step of the convex dual L(lambda) = <w rho exp(phi.lambda), 1> - lambda.target;
    while the moment residual is above 1e-6, a step that would not decrease L is halved
    until it does.  Converged when the
    moment residual is below tol relative to rho (mass, momentum) and to the energy; one
    more full step then takes the multipliers to round-off.

    Inputs over sites (rho, theta [n], u [3, n]); returns (feq [81, n], multipliers [5, n],
    iterations used).  Sites that do not converge within max_iter are NaN."""
    lat = lat or velocity_set()
    rho = np.asarray(rho, dtype=np.float64).reshape(-1)
    th = np.asarray(theta, dtype=np.float64).reshape(-1)
    u1 = np.asarray(u, dtype=np.float64).reshape(3, -1)
    n = rho.size
    phi = np.concatenate([np.ones((lat.q, 1)), lat.c, lat.c2[:, None]], axis=1)      # [81, 5]
    q = (u1 ** 2).sum(axis=0)
    target = np.stack([rho, rho * u1[0], rho * u1[1], rho * u1[2], rho * q + 3.0 * rho * th])  # [5, n]
    scale = np.stack([rho, rho, rho, rho, target[4]])
    lam = np.stack([-1.5 * np.log(th / lat.theta0) - q / (2.0 * th), u1[0] / th, u1[1] / th, u1[2] / th,
                    0.5 / lat.theta0 - 0.5 / th])

    def fdist(l):
        return lat.w[:, None] * rho * np.exp(phi @ l)

    def dual(f, l):
        return f.sum(axis=0) - (l * target).sum(axis=0)

    done = np.zeros(n, dtype=bool)
    failed = np.zeros(n, dtype=bool)
    final = np.zeros(n, dtype=bool)    # converged sites take one more full step
    used = 0
    with np.errstate(over="ignore", invalid="ignore"):
        for it in range(max_iter):
            used = it + 1
            f = fdist(lam)
            r = target - phi.T @ f                                                      # [5, n]
            small = np.all(np.abs(r) <= tol * scale, axis=0)
            done |= final
            final = small & ~done
            active = ~done & ~failed
            if not active.any():
                break
            J = np.einsum("ia,ib,in->nab", phi, phi, f)                                # [n, 5, 5]
            good = np.all(np.isfinite(J), axis=(1, 2)) & (np.abs(np.linalg.det(J)) > 0)
            failed |= active & ~good
            J[~good] = np.eye(5)
            step = np.linalg.solve(J, np.where(good, r, 0.0).T[:, :, None])[:, :, 0].T  # [5, n]
            # full steps once the residual is in Newton's quadratic range (where the dual's
            # decrease is below its own rounding); the safeguard only acts far from it
            near = np.all(np.abs(r) <= 1e-6 * scale, axis=0)
            L0 = dual(f, lam)
            t = np.ones(n)
            for _ in range(60):
                trial = lam + t * step
                Lt = dual(fdist(trial), trial)
                ok = near | (np.isfinite(Lt) & (Lt <= L0 - 1e-4 * t * (r * step).sum(axis=0)))
                if (ok | ~active).all():
                    break
                t = np.where(ok, t, 0.5 * t)
            lam = np.where(active & good, lam + t * step, lam)
    f = fdist(lam)
    f[:, ~done] = np.nan
    return f, lam, used


def boltzmann_h(f: np.ndarray, lat: Lattice | None = None):
    """H = <f, log(f/w) - 1> (Sec. III) per site; f[81, ...] positive."""
    lat = lat or velocity_set()
    w = lat.w.reshape((lat.q,) + (1,) * (np.ndim(f) - 1))
    return (f * (np.log(f / w) - 1.0)).sum(axis=0)


# ---------------------------------------------------------------------------------------
# Streaming on the primary + replica (BCC) lattice, Sec. II Eq. (discretelbm)
# ---------------------------------------------------------------------------------------

def pull_displacement(h: np.ndarray, target_sub: int):
    """Index displacement d (out[n] = src[n - d]) and source sublattice for pulling the
    population with half-unit velocity h into a site of sublattice ``target_sub``.

    A P site with index n sits at n, an R site with index n at n + (1/2, 1/2, 1/2).  The
    population arriving at position p left p - c = p - h/2 one step earlier:
      * h even (integer link): same sublattice, d = h/2;
      * h odd, target P:  source position n - h/2 is the R site with index n - (h+1)/2;
      * h odd, target R:  source position n + 1/2 - h/2 is the P site n - (h-1)/2.
    """
    h = np.asarray(h)
    if np.all(h % 2 == 0):
        return h // 2, target_sub
    if target_sub == 0:
        return (h + 1) // 2, 1
    return (h - 1) // 2, 0


def fill_ghosts_x(fs: np.ndarray, bc_lo, bc_hi, feq_lo=None, feq_hi=None, width: int = 4):
    """Extend one sublattice's populations fs[i, z, y, x] by ``width`` ghost layers at each
    x face.  Returns ext[i, z, y, x + width].

    Boundary kinds (one per face):
      "periodic"      ghosts are the interior layers of the opposite side (wrap-around);
      "zero_gradient" every ghost layer copies all populations of the nearest interior
                      layer of the same sublattice (same y, z) -- an outflow face;
      "eq_inflow"     every ghost site holds feq(rho_in, u_in, theta_in) (``feq_lo`` /
                      ``feq_hi``: the 81 values, identical on both sublattices);
      "bounce_back"   a solid wall: the ghosts are never used (NaN here), ``stream`` returns
                      every population whose link crosses the wall to its own site.
    """
    q, nz, ny, nx = fs.shape
    ext = np.empty((q, nz, ny, nx + 2 * width))
    ext[..., width:width + nx] = fs
    for side, kind, feq in (("lo", bc_lo, feq_lo), ("hi", bc_hi, feq_hi)):
        sl = slice(0, width) if side == "lo" else slice(width + nx, 2 * width + nx)
        if kind == "periodic":
            src = fs[..., nx - width:] if side == "lo" else fs[..., :width]
            if nx < width:  # wrap more than once
                idx = (np.arange(-width, 0) if side == "lo" else np.arange(nx, nx + width)) % nx
                src = fs[..., idx]
            ext[..., sl] = src
        elif kind == "zero_gradient":
            edge = fs[..., 0:1] if side == "lo" else fs[..., nx - 1:nx]
            ext[..., sl] = edge
        elif kind == "eq_inflow":
            ext[..., sl] = np.asarray(feq, dtype=np.float64).reshape(q, 1, 1, 1)
        elif kind == "bounce_back":
            ext[..., sl] = np.nan
        else:
            raise ValueError(f"unknown boundary kind {kind!r}")
    return ext


def stream(f: np.ndarray, bc=("periodic", "periodic"), feq_in=(None, None),
           lat: Lattice | None = None):
    """Pull streaming: f_pre[s, i, n] = f_post[src_sub, i, n - d] for every site of both
    sublattices (left-hand side of Eq. (discretelbm) with dt = 1).

    y and z are periodic; ``bc`` gives the kinds of the -x and +x faces (see
    ``fill_ghosts_x``); ``feq_in`` the inflow populations of those faces (or None).

    A "bounce_back" face is a solid wall (Sec. IV A: the Sod tube's x ends).  The fluid is the
    index range 0 <= x < nx of both sublattices; a population f*_j leaving site n along a link
    whose end has an x index outside that range comes back to n reversed, so
    f_i(n, t + 1) = f*_{-i}(n, t) wherever the source n - d of the pull lies outside.  Every
    population is kept (a permutation of the values), so mass and energy are conserved exactly.
    """
    lat = lat or velocity_set()
    width = 4
    ext = [fill_ghosts_x(f[s], bc[0], bc[1], feq_in[0], feq_in[1], width) for s in (0, 1)]
    nx = f.shape[-1]
    opp = [int(np.flatnonzero(np.all(lat.h == -lat.h[i], axis=1))[0]) for i in range(lat.q)]
    xs = np.arange(nx)
    out = np.empty_like(f)
    for s in (0, 1):
        for i in range(lat.q):
            d, src = pull_displacement(lat.h[i], s)
            dx, dy, dz = (int(v) for v in d)
            a = ext[src][i]                               # [z, y, x + width]
            a = a[:, :, width - dx:width - dx + nx]        # out[x] = ext[x + width - dx]
            a = np.roll(a, shift=(dz, dy), axis=(0, 1))    # out[n] = src[n - d] in y, z
            out[s, i] = a
            # walls: the source x index is x - dx
            cut = ((xs - dx < 0) & (bc[0] == "bounce_back")) | ((xs - dx >= nx) & (bc[1] == "bounce_back"))
            if cut.any():
                out[s, i][..., cut] = f[s, opp[i]][..., cut]
    return out


# ---------------------------------------------------------------------------------------
# Collision, Sec. II Eq. (discretelbm)
# ---------------------------------------------------------------------------------------

def beta_of_tau(tau: float) -> float:
    """beta = dt / (2 tau + dt) with dt = 1 (Sec. II, below Eq. (discretelbm))."""
    return 1.0 / (2.0 * tau + 1.0)


def collide(f: np.ndarray, feq: np.ndarray, tau: float, alpha=2.0) -> np.ndarray:
    """f + alpha beta (feq - f) (Eq. (discretelbm)); alpha = 2 (BGK) or one value per site."""
    return f + np.asarray(alpha) * beta_of_tau(tau) * (feq - f)


def _phi(y):
    """(1 + y) log(1 + y) - y for y >= -1 (its limit 1 at y = -1)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        v = (1.0 + y) * np.log1p(y) - y
    return np.where(y <= -1.0, 1.0, v)


def entropic_delta_h(alpha, f, feq):
    """Delta H(alpha) = H[f + alpha (feq - f)] - H[f] of Eq. (delH), H = <f, log(f/w) - 1>,
    for feq the exact entropic equilibrium of f's own conserved moments.

    With D = feq - f and x = D / f: H[f + alpha D] - H[f] = <alpha D, log(f/w)> +
    <f, (1 + alpha x) log(1 + alpha x) - alpha x>.  Because log(feq / w) = mu + zeta.c + gamma c^2
    and D carries no mass, momentum or energy, <D, log(feq/w)> = 0, so
    <D, log(f/w)> = -<D, log(feq/f)> = -<f, x log(1 + x)>, and

        Delta H(alpha) = <f, (1 + alpha x) log(1 + alpha x) - alpha x> - alpha <f, x log(1 + x)>,

    a sum of terms of order f x^2 with no cancellation between O(1) numbers.  f, feq [81, n]
    (positive), alpha scalar or [n]."""
    x = (feq - f) / f
    b = (f * x * np.log1p(x)).sum(axis=0)
    return (f * _phi(np.asarray(alpha) * x)).sum(axis=0) - np.asarray(alpha) * b


def entropic_alpha(f, feq, max_iter: int = 200):
    """Entropic alpha (Sec. II, Eq. (delH)): the nontrivial root alpha > 0 of
    H[f + alpha (feq - f)] - H[f] = 0, per site, with feq the exact entropic equilibrium.

    Along the line f + alpha D, Delta H is convex, zero at alpha = 0, falls at first (at alpha = 1
    it is H[feq] - H[f] < 0), so it has exactly one positive root where it rises through zero,
    provided the root lies where every population stays positive, alpha < alpha_max =
    min over D_i < 0 of f_i / (-D_i).
    * Newton from alpha = 2 when Delta H(2) > 0: for a convex function started right of its
      root the iterates decrease monotonically to it.  Stops when a step is below 1e-15 alpha.
    * otherwise the root lies above 2: bisection on [1, alpha_max] (or on [1, hi] with hi
      doubled from 2 until Delta H(hi) > 0), 200 halvings.
    * no sign change up to alpha_max: alpha = alpha_max (the furthest positive state on the line).
    * f = feq (no deviation): alpha = 2, the limit of the root as D -> 0.
    * some f_i <= 0 (H undefined): alpha = 2.
    f, feq [81, n]; returns alpha [n]."""
    f = np.asarray(f, dtype=np.float64)
    feq = np.asarray(feq, dtype=np.float64)
    n = f.shape[1]
    alpha = np.full(n, 2.0)
    pos = np.all(f > 0, axis=0)
    D = feq - f
    with np.errstate(divide="ignore", invalid="ignore"):
        x = np.where(pos, D / np.where(pos, f, 1.0), 0.0)
        amax = np.where(x < 0, -1.0 / np.where(x < 0, x, -1.0), np.inf).min(axis=0)
    b = (f * x * np.log1p(x)).sum(axis=0)
    live = pos & (b > 0)
    if not live.any():
        return alpha

    def F(a, k):
        return (f[:, k] * _phi(a * x[:, k])).sum(axis=0) - a * b[k]

    def dF(a, k):
        return (f[:, k] * x[:, k] * np.log1p(a * x[:, k])).sum(axis=0) - b[k]

    k_all = np.nonzero(live)[0]
    newton = np.zeros(n, dtype=bool)
    ok2 = amax[k_all] > 2.0
    f2 = np.full(k_all.size, -1.0)
    f2[ok2] = F(2.0, k_all[ok2])
    newton[k_all[f2 > 0]] = True
    # Newton from 2 (monotone from the right)
    k = np.nonzero(newton)[0]
    a = np.full(k.size, 2.0)
    act = np.ones(k.size, dtype=bool)
    for _ in range(max_iter):
        if not act.any():
            break
        kk = k[act]
        step = F(a[act], kk) / dF(a[act], kk)
        a[act] -= step
        act[act] = np.abs(step) > 1e-15 * a[act]
    alpha[k] = a
    # bisection above 2
    k = k_all[~newton[k_all]]
    if k.size:
        lo = np.ones(k.size)
        hi = np.where(np.isfinite(amax[k]), amax[k], 2.0)
        grow = ~np.isfinite(amax[k])
        for _ in range(60):
            if not grow.any():
                break
            up = grow & (F(hi, k) <= 0)
            hi = np.where(up, 2.0 * hi, hi)
            grow = up
        root = F(hi, k) > 0
        for _ in range(max_iter):
            mid = 0.5 * (lo + hi)
            neg = F(mid, k) <= 0
            lo = np.where(neg, mid, lo)
            hi = np.where(neg, hi, mid)
        alpha[k] = np.where(root, 0.5 * (lo + hi), np.where(np.isfinite(amax[k]), amax[k], 2.0))
    return alpha


# ---------------------------------------------------------------------------------------
# Whole steps
# ---------------------------------------------------------------------------------------

def init(rho: np.ndarray, u: np.ndarray, theta: np.ndarray, lat: Lattice | None = None,
         chunk: int = 1024, eq: str = "series"):
    """Populations f[s, i, z, y, x] = feq(rho, u, theta) at every site of both sublattices.

    rho, theta: [2, nz, ny, nx]; u: [3, 2, nz, ny, nx]."""
    lat = lat or velocity_set()
    eqf = _equilibrium_of(eq)
    rho = np.asarray(rho, dtype=np.float64)
    S = rho.shape
    r1 = rho.reshape(-1)
    t1 = np.asarray(theta, dtype=np.float64).reshape(-1)
    u1 = np.asarray(u, dtype=np.float64).reshape(3, -1)
    out = np.empty((lat.q, r1.size))
    for a in range(0, r1.size, chunk):
        b = min(a + chunk, r1.size)
        out[:, a:b] = eqf(r1[a:b], u1[:, a:b], t1[a:b], lat)
    return np.moveaxis(out.reshape((lat.q,) + S), 0, 1).copy()


def bc_feq(bc_spec, lat: Lattice | None = None, eq: str = "series"):
    """81 inflow populations of an "eq_inflow" face spec ("eq_inflow", rho, ux, uy, uz, theta),
    else None."""
    if bc_spec[0] != "eq_inflow":
        return None
    _, r, ux, uy, uz, t = bc_spec
    return _equilibrium_of(eq)(np.array([r]), np.array([[ux], [uy], [uz]]), np.array([t]), lat)[:, 0]


def _equilibrium_of(kind: str):
    if kind == "series":
        return equilibrium
    if kind == "series_exact_w":
        return lambda rho, u, theta, lat=None: equilibrium(rho, u, theta, lat, weights="exact")
    if kind == "entropic":
        return lambda rho, u, theta, lat=None: entropic_equilibrium(rho, u, theta, lat)[0].reshape(
            (81,) + np.shape(rho))
    raise ValueError(kind)


def step(f: np.ndarray, tau: float, bc_x=(("periodic",), ("periodic",)),
         lat: Lattice | None = None, chunk: int = 1024, eq: str = "series",
         collision: str = "bgk") -> np.ndarray:
    """One time step: boundary fill, pull streaming, moments, equilibrium, collision.

    ``bc_x`` holds the -x and +x face specs: ("periodic",), ("zero_gradient",),
    ("bounce_back",) or ("eq_inflow", rho, ux, uy, uz, theta).  ``eq`` selects the equilibrium: "series" (App. B)
    or "entropic" (the exact minimiser of Sec. III).  ``collision`` is "bgk" (alpha = 2) or
    "entropic" (alpha the root of Eq. (delH) per site; needs eq="entropic")."""
    lat = lat or velocity_set()
    if collision not in ("bgk", "entropic"):
        raise ValueError(collision)
    if collision == "entropic" and eq != "entropic":
        raise ValueError("the entropic alpha is defined with the entropic equilibrium")
    eqf = _equilibrium_of(eq)
    kinds = (bc_x[0][0], bc_x[1][0])
    if (kinds[0] == "periodic") != (kinds[1] == "periodic"):
        raise ValueError("a periodic x face must be paired with a periodic x face")
    feq_in = (bc_feq(bc_x[0], lat, eq), bc_feq(bc_x[1], lat, eq))
    pre = stream(f, kinds, feq_in, lat)
    flat = np.moveaxis(pre, 1, 0).reshape(lat.q, -1)     # [81, sites]
    post = np.empty_like(flat)
    for a in range(0, flat.shape[1], chunk):
        b = min(a + chunk, flat.shape[1])
        rho, u, theta = moments(flat[:, a:b], lat)
        feq = eqf(rho, u, theta, lat)
        alpha = entropic_alpha(flat[:, a:b], feq) if collision == "entropic" else 2.0
        post[:, a:b] = collide(flat[:, a:b], feq, tau, alpha)
    return np.moveaxis(post.reshape((lat.q,) + f.shape[:1] + f.shape[2:]), 0, 1).copy()


def run(f: np.ndarray, tau: float, nsteps: int, bc_x=(("periodic",), ("periodic",)),
        lat: Lattice | None = None, eq: str = "series", collision: str = "bgk") -> np.ndarray:
    for _ in range(nsteps):
        f = step(f, tau, bc_x, lat, eq=eq, collision=collision)
    return f


def fields(f: np.ndarray, lat: Lattice | None = None):
    """(rho[2,z,y,x], u[3,2,z,y,x], theta[2,z,y,x]) of stored populations f[s, i, z, y, x]."""
    lat = lat or velocity_set()
    return moments(np.moveaxis(f, 1, 0), lat)


def _central_diff(a: np.ndarray, axis: int, periodic: bool) -> np.ndarray:
    """d a / d(index) along ``axis`` by second-order central differences (unit spacing);
    on a non-periodic axis the two end planes take second-order one-sided differences."""
    if periodic:
        return 0.5 * (np.roll(a, -1, axis=axis) - np.roll(a, 1, axis=axis))
    a = np.moveaxis(a, axis, 0)
    d = np.empty_like(a)
    d[1:-1] = 0.5 * (a[2:] - a[:-2])
    d[0] = -1.5 * a[0] + 2.0 * a[1] - 0.5 * a[2]
    d[-1] = 1.5 * a[-1] - 2.0 * a[-2] + 0.5 * a[-3]
    return np.moveaxis(d, 0, axis)


def diagnostics(f: np.ndarray, lat: Lattice | None = None, x_periodic: bool = True):
    """Mean kinetic energy and mean enstrophy of Sec. IV C (compressible Taylor-Green vortex):

        KE = (1/|Omega|) int rho u.u / 2 dOmega,   eps = (1/|Omega|) int rho w.w / 2 dOmega,
        w = curl u,

    as averages over all sites of both sublattices.  The paper gives no discretisation of the
    curl; here each sublattice is differentiated on its own grid (unit spacing, second-order
    central differences; y and z periodic, x periodic or with one-sided second-order end
    differences).  f[s, i, z, y, x]; returns (KE, eps)."""
    rho, u, _ = fields(f, lat)                          # rho[s,z,y,x], u[a,s,z,y,x]
    ke = (0.5 * rho * (u ** 2).sum(axis=0)).mean()
    # axis of u[a] arrays: s=0, z=1, y=2, x=3
    d = lambda comp, ax: _central_diff(u[comp], {"x": 3, "y": 2, "z": 1}[ax], x_periodic or ax != "x")
    wx = d(2, "y") - d(1, "z")
    wy = d(0, "z") - d(2, "x")
    wz = d(1, "x") - d(0, "y")
    ens = (0.5 * rho * (wx ** 2 + wy ** 2 + wz ** 2)).mean()
    return float(ke), float(ens)


def totals(f: np.ndarray, lat: Lattice | None = None):
    """Global sums (sum rho, sum rho u_x, sum rho u_y, sum rho u_z, sum <f, c^2>) over all
    sites: the conserved quantities of Eq. (conslaws) summed over the grid."""
    lat = lat or velocity_set()
    g = np.moveaxis(f, 1, 0).reshape(lat.q, -1).sum(axis=1)
    return np.array([g.sum(), *(lat.c.T @ g), lat.c2 @ g])
