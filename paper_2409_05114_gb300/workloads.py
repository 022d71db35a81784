"""Seeded synthetic initial conditions for the RD3Q81 step.

This module only builds macroscopic initial fields (rho, u, theta) on the primary +
replica lattice and the boundary specification of each workload.  It holds none of the
method's arithmetic (no equilibrium, no streaming, no collision), so the CUDA path and the
FP64 oracle can both start from exactly the same inputs.

Field layout (the library's): arrays of shape [2, nz, ny, nx] (sublattice P then R; P site
n sits at position n, R site n at n + 1/2), velocity [3, 2, nz, ny, nx]; flattening gives
the C-ABI's site-major order.

Workloads (sizes and parameters of the paper's benchmarks, Sec. IV):
  sod            Sod-type shock tube along x, zero-gradient x faces
  taylor_green   compressible Taylor-Green vortex (Sec. IV C initial field)
  hit            decaying isotropic turbulence, random-phase solenoidal field
  mach2_blob     Mach-2 uniform flow with a density blob and an isentropic vortex,
                 equilibrium inflow at -x, zero-gradient outflow at +x
Relaxation times are given in the conventional LB form tau_lb (omega = 1/tau_lb); the
paper's tau (beta = 1/(2 tau + 1), so omega = 2 beta) is tau_lb - 1/2.  ``paper_tau``
converts; with ``reading="literal"`` the listed value is used as the paper's tau directly.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

THETA0 = 0.821035006329447750282591763   # reference temperature of RD3Q81 (Table "tab:weights")
GAMMA = 5.0 / 3.0                         # monatomic gas: E = rho u^2 + 3 rho theta
CS = float(np.sqrt(GAMMA * THETA0))       # adiabatic sound speed sqrt(gamma theta0), Sec. IV C


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    tau_lb: float
    steps: int
    rho: np.ndarray
    u: np.ndarray
    theta: np.ndarray
    faces: list = field(default_factory=lambda: ["periodic"] * 6)
    note: str = ""

    @property
    def sites(self) -> int:
        return 2 * self.nx * self.ny * self.nz

    def paper_tau(self, reading: str = "lb") -> float:
        return paper_tau(self.tau_lb, reading)

    def oracle_bc_x(self):
        def conv(spec):
            return (spec,) if isinstance(spec, str) else tuple(spec)
        return conv(self.faces[0]), conv(self.faces[1])


def paper_tau(tau_listed: float, reading: str = "lb") -> float:
    """Paper tau from a listed relaxation time: "lb" reads it as tau_lb (tau = tau_lb - 1/2),
    "literal" as the paper's tau itself."""
    if reading == "lb":
        return tau_listed - 0.5
    if reading == "literal":
        return tau_listed
    raise ValueError(reading)


def positions(nx: int, ny: int, nz: int):
    """Physical positions (x, y, z), each [2, nz, ny, nx]: P at n, R at n + 1/2."""
    z, y, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float),
                          np.arange(nx, dtype=float), indexing="ij")
    return tuple(np.stack([a, a + 0.5]) for a in (x, y, z))


def sod(nx: int = 512, ny: int = 4, nz: int = 4, tau_lb: float = 0.6, steps: int = 200,
        walls: bool = False) -> Workload:
    """Left half rho = 1, theta = theta0; right half rho = 0.125, theta = 0.8 theta0; u = 0.
    The interface is at x = nx/2 (physical position).  x faces zero-gradient, or with ``walls``
    bounce-back as in the paper's Sod setup (Sec. IV A: 4000 x 8 x 8, periodic y and z)."""
    x, _, _ = positions(nx, ny, nz)
    left = x < nx / 2.0
    rho = np.where(left, 1.0, 0.125)
    theta = np.where(left, THETA0, 0.8 * THETA0)
    u = np.zeros((3,) + rho.shape)
    x_face = "bounce_back" if walls else "zero_gradient"
    return Workload("sod_walls" if walls else "sod", nx, ny, nz, tau_lb, steps, rho, u, theta,
                    [x_face, x_face] + ["periodic"] * 4)


def shock_tube(nx: int = 512, ny: int = 4, nz: int = 4, rho_right: float = 0.125, theta_right: float = 0.8,
               tau_lb: float = 0.6, steps: int = 200, walls: bool = False) -> Workload:
    """Sod-type tube: left rho = 1, theta = theta0; right rho = rho_right,
    theta = theta_right * theta0; u = 0; interface at x = nx/2; zero-gradient x faces, or
    bounce-back walls with ``walls``."""
    wl = sod(nx, ny, nz, tau_lb, steps, walls)
    x, _, _ = positions(nx, ny, nz)
    left = x < nx / 2.0
    wl.rho = np.where(left, 1.0, rho_right)
    wl.theta = np.where(left, THETA0, theta_right * THETA0)
    wl.name = f"shock_tube_{nx}_r{rho_right:g}_t{theta_right:g}"
    return wl


def taylor_green(n: int = 128, mach: float = 0.5, tau_lb: float = 0.51, steps: int = 1000) -> Workload:
    """u = U0 (sin x^ cos y^ cos z^, -cos x^ sin y^ cos z^, 0), rho = 1,
    p = p0 + rho0 U0^2/16 (cos 2x^ + cos 2y^)(cos 2z^ + 2) with p0 = theta0 and theta = p/rho,
    x^ = 2 pi x / n, U0 = mach * c_s."""
    x, y, z = positions(n, n, n)
    k = 2.0 * np.pi / n
    X, Y, Z = k * x, k * y, k * z
    U0 = mach * CS
    u = np.stack([U0 * np.sin(X) * np.cos(Y) * np.cos(Z), -U0 * np.cos(X) * np.sin(Y) * np.cos(Z), np.zeros_like(X)])
    rho = np.ones_like(X)
    theta = THETA0 + U0 ** 2 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    return Workload(f"taylor_green_{n}", n, n, n, tau_lb, steps, rho, u, theta)


def hit(n: int = 256, mach_rms: float = 0.5, seed: int = 2409, tau_lb: float = 0.505, steps: int = 500) -> Workload:
    """Random-phase solenoidal velocity with energy spectrum E(k) ~ k^4 exp(-2 (k/4)^2),
    scaled so that sqrt(<|u|^2>) over all sites = mach_rms * c_s; rho = 1, theta = theta0.
    The Fourier series is evaluated exactly on both sublattices (the replica sites by a
    half-cell phase shift); Nyquist modes are zero."""
    rng = np.random.default_rng(seed)
    kk = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")
    K2 = KX ** 2 + KY ** 2 + KZ ** 2
    Kmag = np.sqrt(K2)
    spec = Kmag ** 4 * np.exp(-2.0 * (Kmag / 4.0) ** 2)
    amp = np.zeros_like(Kmag)
    nz_ = K2 > 0
    amp[nz_] = np.sqrt(spec[nz_] / (4.0 * np.pi * K2[nz_]))
    nyq = (np.abs(KX) == n // 2) | (np.abs(KY) == n // 2) | (np.abs(KZ) == n // 2)
    amp[nyq] = 0.0
    a = (rng.normal(size=(3, n, n, n)) + 1j * rng.normal(size=(3, n, n, n))) * amp
    # solenoidal projection: a - k (k . a) / |k|^2
    kdot = KX * a[0] + KY * a[1] + KZ * a[2]
    with np.errstate(invalid="ignore", divide="ignore"):
        kd = np.where(nz_, kdot / np.where(nz_, K2, 1.0), 0.0)
    a = a - np.stack([KX, KY, KZ]) * kd
    # Hermitian-symmetric field: take the real part of the complex synthesis
    shift = np.exp(2j * np.pi * (KX + KY + KZ) * 0.5 / n)
    uP = np.real(np.fft.ifftn(a, axes=(1, 2, 3)))
    uR = np.real(np.fft.ifftn(a * shift, axes=(1, 2, 3)))
    u = np.stack([uP, uR], axis=1)                      # [3, 2, z, y, x]
    rms = np.sqrt((u ** 2).sum(axis=0).mean())
    u *= mach_rms * CS / rms
    rho = np.ones((2, n, n, n))
    theta = np.full_like(rho, THETA0)
    return Workload(f"hit_{n}", n, n, n, tau_lb, steps, rho, u, theta)


def mach2_blob(nx: int = 1024, ny: int = 256, nz: int = 4, seed: int = 5114, tau_lb: float = 0.55,
               steps: int = 2000, blob_amp: float = 0.2, sigma: float = 16.0, vortex: float = 0.3,
               radius: float = 16.0, mach: float = 2.0) -> Workload:
    """Uniform Mach-2 flow in x (U = mach c_s, mach = 2; rho = 1, theta = theta0), a Gaussian density blob
    (amplitude 0.2, sigma 16 cells, centre drawn from the seed near (nx/4, ny/2)) and an
    isentropic vortex at (nx/4, ny/2): u_phi = eps U (r/R) exp((1 - r^2/R^2)/2),
    theta = theta0 - (2/5) (eps U)^2 / 2 exp(1 - r^2/R^2), rho ~ (theta/theta0)^(3/2).
    Equilibrium inflow of the free stream at -x, zero-gradient outflow at +x."""
    rng = np.random.default_rng(seed)
    x, y, _ = positions(nx, ny, nz)
    U = mach * CS
    xc, yc = nx / 4.0, ny / 2.0
    bx, by = xc + rng.uniform(-8, 8), yc + rng.uniform(-8, 8)
    dx, dy = x - xc, y - yc
    r2 = (dx ** 2 + dy ** 2) / radius ** 2
    uphi_over_r = vortex * U / radius * np.exp((1.0 - r2) / 2.0)
    ux = U - uphi_over_r * dy
    uy = uphi_over_r * dx
    theta = THETA0 - 0.4 * (vortex * U) ** 2 / 2.0 * np.exp(1.0 - r2)
    blob = 1.0 + blob_amp * np.exp(-((x - bx) ** 2 + (y - by) ** 2) / (2.0 * sigma ** 2))
    rho = (theta / THETA0) ** 1.5 * blob
    u = np.stack([ux, uy, np.zeros_like(ux)])
    faces = [("eq_inflow", 1.0, U, 0.0, 0.0, THETA0), "zero_gradient"] + ["periodic"] * 4
    name = f"mach2_blob_{nx}x{ny}x{nz}" if mach == 2.0 else f"blob_mach{mach:g}_{nx}x{ny}x{nz}"
    return Workload(name, nx, ny, nz, tau_lb, steps, rho, u, theta, faces)


def smooth_random(nx: int, ny: int, nz: int, seed: int = 0, mach: float = 0.3, eta: float = 0.05,
                  tau_lb: float = 0.6, steps: int = 10, faces=None) -> Workload:
    """Small smooth periodic perturbation (a few random Fourier modes) for parity tests."""
    rng = np.random.default_rng(seed)
    x, y, z = positions(nx, ny, nz)
    def mode():
        kx, ky, kz = (rng.integers(1, 3) * 2 * np.pi / m for m in (nx, ny, nz))
        ph = rng.uniform(0, 2 * np.pi, 3)
        return np.sin(kx * x + ph[0]) * np.cos(ky * y + ph[1]) * np.cos(kz * z + ph[2])
    rho = 1.0 + 0.05 * mode()
    theta = THETA0 * (1.0 + eta * mode())
    u = np.stack([mach * CS * mode(), mach * CS * mode(), 0.5 * mach * CS * mode()])
    return Workload(f"smooth_{nx}x{ny}x{nz}", nx, ny, nz, tau_lb, steps, rho, u, theta,
                    faces or ["periodic"] * 6)


@dataclass
class ServedRequest:
    workload: Workload
    storage: str
    nsteps: int
    arrival_s: float
    tau: float           # the paper's tau passed to the library
    equilibrium: str = "entropic"
    family: str = ""


def tgv_served_tau(n: int, mach: float, reynolds: float = 400.0, tau_min: float = 0.05) -> float:
    """Paper tau of a served Taylor-Green case: the viscosity nu = tau theta0 (Sec. II) that gives
    Re = U0 L / nu with L = n / (2 pi) (the field's length scale) and U0 = mach c_s, at the
    Reynolds number of the paper's Mach-1 run (Sec. IV C: Re 400), but no lower than tau_min
    (tau_lb 0.55)."""
    u0 = mach * CS
    return max(tau_min, u0 * (n / (2.0 * np.pi)) / (reynolds * THETA0))


def served_mix(n_requests: int = 128, seed: int = 5114, mean_interarrival_s: float = 0.03,
               max_steps: int = 2000) -> list:
    """Mixed-size request stream (seeded; the served-batch workload): Poisson arrivals, each
    request drawn uniformly from three families:
      * Sod-type shock tubes nx x 4 x 4, nx in {256, 512, 1024, 2048}: rho 1 | 0.125, theta
        theta0 | 0.8 theta0, zero-gradient x faces, tau_lb 0.6 (the shock-tube workload);
      * Taylor-Green vortices n^3, n in {32, 48, 64, 96, 128, 160, 192}, Ma in {0.3, 0.5, 0.7,
        1.0}, tau from tgv_served_tau (Re 400, at least tau_lb 0.55);
      * Mach-2 blob flows (blob, isentropic vortex, inflow / outflow) on 256x256x4, 512x128x4,
        512x256x4 and 1024x256x4, tau_lb 0.55 (the Mach-2 workload);
    each with 200 .. max_steps steps, FP32 or FP16-offset storage (even odds) and the exact
    entropic equilibrium of Sec. III, with which every member of these families runs its 2000
    steps (the series equilibrium fails on the Mach-2 blobs at once, on Mach-1 vortices and on
    the strong Sod tube within a few hundred steps).  Field generation is cached per shape."""
    rng = np.random.default_rng(seed)
    cache = {}
    out = []
    t = 0.0
    for _ in range(n_requests):
        t += rng.exponential(mean_interarrival_s)
        fam = int(rng.integers(0, 3))
        if fam == 0:
            nx = int(rng.choice([256, 512, 1024, 2048]))
            key = ("tube", nx)
            if key not in cache:
                cache[key] = sod(nx=nx)
            wl, tau, name = cache[key], paper_tau(0.6, "lb"), "shock_tube"
        elif fam == 1:
            n = int(rng.choice([32, 48, 64, 96, 128, 160, 192]))
            ma = float(rng.choice([0.3, 0.5, 0.7, 1.0]))
            key = ("tgv", n, ma)
            if key not in cache:
                cache[key] = taylor_green(n, mach=ma)
            wl, tau, name = cache[key], tgv_served_tau(n, ma), "taylor_green"
        else:
            shape = [(256, 256, 4), (512, 128, 4), (512, 256, 4), (1024, 256, 4)][int(rng.integers(0, 4))]
            key = ("blob",) + shape
            if key not in cache:
                cache[key] = mach2_blob(*shape)
            wl, tau, name = cache[key], paper_tau(0.55, "lb"), "mach2_blob"
        steps = int(rng.integers(200, max_steps + 1))
        storage = "f32" if rng.random() < 0.5 else "f16"
        out.append(ServedRequest(wl, storage, steps, t, tau, "entropic", name))
    return out
