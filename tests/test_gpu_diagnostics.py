"""GPU kinetic energy and enstrophy (lbm_diagnostics, Sec. IV C) against the oracle's and
against the closed form of a sampled TGV velocity field (rho = 1):
KE = U0^2 / 8, eps = (3/8) U0^2 sin^2(2 pi / N).  Tolerances: FP64 storage 1e-12 relative
(identical arithmetic up to summation order); FP32 storage 1e-6 (the stored populations)."""

import numpy as np
import pytest

from parity_util import ensure_built, gpu_run, oracle_run
from oracle import rd3q81 as O
from paper_2409_05114_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2409_05114_gb300 import binding
    return binding


def _diag(B, wl, steps, tau, storage, eq="series"):
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, storage, wl.faces, equilibrium=eq)
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_init(ctx, np.ascontiguousarray(wl.rho, dtype=np.float64).reshape(-1),
                   np.ascontiguousarray(wl.u, dtype=np.float64).reshape(-1),
                   np.ascontiguousarray(wl.theta, dtype=np.float64).reshape(-1))
        B.lbm_step(ctx, steps)
        return B.lbm_diagnostics(ctx)
    finally:
        B.lbm_destroy(ctx)


def test_closed_form_tgv_velocity(B):
    N, U0 = 16, 0.1
    wl = W.taylor_green(N, mach=0.5)
    s = np.arange(2)[:, None, None, None] * 0.5
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    X, Y, Z = (2 * np.pi * (q + s) / N for q in (x, y, z))
    wl.u = np.stack([U0 * np.sin(X) * np.cos(Y) * np.cos(Z), -U0 * np.cos(X) * np.sin(Y) * np.cos(Z), 0 * X])
    wl.rho = np.ones_like(X)
    wl.theta = np.full_like(X, W.THETA0)
    ke, ens = _diag(B, wl, 0, 0.01, "f64")
    assert ke == pytest.approx(U0 ** 2 / 8, rel=1e-12)
    assert ens == pytest.approx(3 / 8 * U0 ** 2 * np.sin(2 * np.pi / N) ** 2, rel=1e-12)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_tgv_after_steps_matches_oracle(B, storage, tol):
    wl = W.taylor_green(16, mach=0.5)
    tau = wl.paper_tau("lb")
    ref = O.diagnostics(oracle_run(wl, 10, tau))
    got = _diag(B, wl, 10, tau, storage)
    print("diagnostics %s TGV16 10 steps: KE %.9g (oracle %.9g), eps %.9g (oracle %.9g)" % (storage, got[0], ref[0], got[1], ref[1]))
    np.testing.assert_allclose(got, ref, rtol=tol)


def test_non_periodic_x_matches_oracle(B):
    wl = W.mach2_blob(32, 8, 4, mach=0.5, vortex=0.1)
    tau = wl.paper_tau("literal")
    ref = O.diagnostics(oracle_run(wl, 5, tau), x_periodic=False)
    got = _diag(B, wl, 5, tau, "f64")
    np.testing.assert_allclose(got, ref, rtol=1e-12)
