"""Helpers shared by the parity tests: run a workload through the CUDA library (C-ABI via
the binding) and through the FP64 oracle on the same seeded inputs, and compare."""

from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import rd3q81 as O  # noqa: E402


def ensure_built():
    lib = os.path.join(ROOT, "paper_2409_05114_gb300", "liblbm_rd3q81.so")
    if not os.path.exists(lib):
        from paper_2409_05114_gb300 import build_lib
        build_lib.build()
    return lib


def lib_perm():
    """perm[i] = oracle direction index of library direction i."""
    from paper_2409_05114_gb300 import binding as B
    h, _ = B.lbm_velocities()
    idx = {tuple(v): k for k, v in enumerate(O.velocity_set().h)}
    return np.array([idx[tuple(int(x) for x in v)] for v in h])


def oracle_run(wl, steps: int, tau: float, eq: str = "series", collision: str = "bgk"):
    f = O.init(wl.rho, wl.u, wl.theta, eq=eq)
    f = O.run(f, tau, steps, wl.oracle_bc_x(), eq=eq, collision=collision)
    return f


def gpu_run(wl, steps: int, tau: float, storage: str, fp64_moments=False, populations=None, eq="series",
            check_stable=False, collision="bgk"):
    """Returns (f_lib[2, 81, z, y, x] in library order, rho, u, theta) after `steps`."""
    from paper_2409_05114_gb300 import binding as B
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, storage, wl.faces, fp64_moments, equilibrium=eq,
                        collision=collision)
    ctx = B.lbm_create(cfg)
    try:
        if populations is None:
            B.lbm_init(ctx, np.ascontiguousarray(wl.rho, dtype=np.float64).reshape(-1),
                       np.ascontiguousarray(wl.u, dtype=np.float64).reshape(-1),
                       np.ascontiguousarray(wl.theta, dtype=np.float64).reshape(-1))
        else:
            B.lbm_set_populations(ctx, np.ascontiguousarray(populations).reshape(-1))
        B.lbm_step(ctx, steps)
        if check_stable:
            B.lbm_sync(ctx)
        S = wl.sites
        rho, u, th = np.zeros(S), np.zeros(3 * S), np.zeros(S)
        B.lbm_moments(ctx, rho, u, th)
        f = np.zeros(2 * 81 * wl.nx * wl.ny * wl.nz)
        B.lbm_get_populations(ctx, f)
    finally:
        B.lbm_destroy(ctx)
    shp = (2, wl.nz, wl.ny, wl.nx)
    return f.reshape((2, 81) + shp[1:]), rho.reshape(shp), u.reshape((3,) + shp), th.reshape(shp)


def to_library_order(f_oracle, perm):
    return f_oracle[:, perm]


def field_errors(ref, got):
    """Max relative errors (rho, u, theta): rho and theta pointwise |d|/|ref|; u as
    max |du| / max |u_ref| (u crosses zero)."""
    (r0, u0, t0), (r1, u1, t1) = ref, got
    er = np.max(np.abs(r1 - r0) / np.abs(r0))
    et = np.max(np.abs(t1 - t0) / np.abs(t0))
    umax = np.max(np.abs(u0))
    eu = np.max(np.abs(u1 - u0)) / (umax if umax > 0 else 1.0)
    return float(er), float(eu), float(et)


def population_error(f_ref_lib_order, f_got, w_lib):
    """max |df_i| / w_i over all sites and directions (populations scale with w_i)."""
    return float(np.max(np.abs(f_got - f_ref_lib_order) / w_lib.reshape(1, 81, 1, 1, 1)))


def site_coords(wl, sites):
    n = wl.nx * wl.ny * wl.nz
    sites = np.asarray(sites, dtype=np.int64)
    sub, t = sites // n, sites % n
    return sub, t % wl.nx, (t // wl.nx) % wl.ny, t // (wl.nx * wl.ny)


def oracle_sampled_step(wl, sites, tau, eq="series", collision="bgk", store=None):
    """One step of the oracle at selected sites of a periodic grid, computed site by site
    from the initial state f = feq(fields) (App. B series, or the exact entropic equilibrium
    with eq="entropic"): each target pulls its 81 populations from the equilibria of its source
    sites (index maps of oracle.pull_displacement), then moments, equilibrium and collision (BGK,
    or the entropic alpha of Eq. (delH) with collision="entropic").  store(f [81, U]), if given,
    maps the initial populations to the values a storage format holds.  Returns post-collision
    populations [81, K], oracle order."""
    assert all((f if isinstance(f, str) else f[0]) == "periodic" for f in wl.faces)
    lat = O.velocity_set()
    feq_of = (lambda r, u, t: O.entropic_equilibrium(r, u, t, lat)[0]) if eq == "entropic" else O.equilibrium
    n = wl.nx * wl.ny * wl.nz
    sub, x, y, z = site_coords(wl, sites)
    src = np.empty((lat.q, len(sub)), dtype=np.int64)
    for i in range(lat.q):
        for s in (0, 1):
            d, ss = O.pull_displacement(lat.h[i], s)
            m = sub == s
            sx = (x[m] - d[0]) % wl.nx
            sy = (y[m] - d[1]) % wl.ny
            sz = (z[m] - d[2]) % wl.nz
            src[i, m] = ss * n + (sz * wl.ny + sy) * wl.nx + sx
    uniq, inv = np.unique(src, return_inverse=True)
    inv = inv.reshape(src.shape)
    rho = wl.rho.reshape(-1)[uniq]
    u = wl.u.reshape(3, -1)[:, uniq]
    th = wl.theta.reshape(-1)[uniq]
    feq_src = feq_of(rho, u, th)                            # [81, U]
    if store is not None:
        feq_src = store(feq_src)
    pulled = feq_src[np.arange(lat.q)[:, None], inv]        # [81, K]
    r, uu, t = O.moments(pulled)
    feq = feq_of(r, uu, t)
    alpha = O.entropic_alpha(pulled, feq) if collision == "entropic" else 2.0
    return O.collide(pulled, feq, tau, alpha=alpha)
