"""The seeded input generators: deterministic, the shapes and statistics their docstrings
state (solenoidal HIT at the requested rms Mach, TGV initial field, blob inflow state), and
the served mix's request stream."""

import numpy as np

from paper_2409_05114_gb300 import workloads as W


def test_hit_solenoidal_rms_and_deterministic():
    a = W.hit(16, seed=2409)
    b = W.hit(16, seed=2409)
    np.testing.assert_array_equal(a.u, b.u)
    assert not np.array_equal(a.u, W.hit(16, seed=1).u)
    assert abs(np.sqrt((a.u ** 2).sum(0).mean()) / W.CS - 0.5) < 1e-12
    n = 16
    k = np.fft.fftfreq(n, 1.0 / n) * 2 * np.pi / n
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    for s in (0, 1):
        u = a.u[:, s]
        div = np.fft.ifftn(1j * (KX * np.fft.fftn(u[0]) + KY * np.fft.fftn(u[1]) + KZ * np.fft.fftn(u[2])))
        assert np.abs(div).max() < 1e-12
    assert np.all(a.rho == 1.0) and np.all(a.theta == W.THETA0)


def test_taylor_green_fields():
    wl = W.taylor_green(8, mach=0.5)
    x, y, z = W.positions(8, 8, 8)
    X, Y, Z = (2 * np.pi * v / 8 for v in (x, y, z))
    U0 = 0.5 * W.CS
    np.testing.assert_allclose(wl.u[0], U0 * np.sin(X) * np.cos(Y) * np.cos(Z), atol=1e-15)
    assert np.all(wl.u[2] == 0)
    # mean temperature is theta0 (the cosine products average to zero over a period)
    assert abs(wl.theta.mean() - W.THETA0) < 1e-12
    assert wl.sites == 2 * 8 ** 3


def test_blob_inflow_state_is_free_stream():
    wl = W.mach2_blob(256, 64, 4)
    kind, rho, ux, uy, uz, th = wl.faces[0]
    assert kind == "eq_inflow" and rho == 1.0 and abs(ux - 2 * W.CS) < 1e-15 and th == W.THETA0
    assert wl.faces[1] == "zero_gradient"
    # far from the blob and the vortex the flow is the free stream
    np.testing.assert_allclose(wl.u[0][:, :, :, -1], 2 * W.CS, rtol=1e-6)


def test_sod_and_tau_readings():
    wl = W.sod(64, 2, 2)
    assert wl.rho[0, 0, 0, 0] == 1.0 and wl.rho[0, 0, 0, -1] == 0.125
    assert abs(wl.paper_tau("lb") - 0.1) < 1e-15 and wl.paper_tau("literal") == 0.6


def test_served_mix_deterministic():
    a = W.served_mix(24, seed=5114)
    b = W.served_mix(24, seed=5114)
    assert [(r.workload.name, r.storage, r.nsteps, r.arrival_s, r.tau) for r in a] == \
           [(r.workload.name, r.storage, r.nsteps, r.arrival_s, r.tau) for r in b]
    assert all(200 <= r.nsteps <= 2000 and r.storage in ("f32", "f16") for r in a)
    assert all(x.arrival_s < y.arrival_s for x, y in zip(a, a[1:]))
    assert {r.family for r in a} == {"shock_tube", "taylor_green", "mach2_blob"}
    assert all(r.equilibrium == "entropic" for r in a)
    for r in a:
        wl = r.workload
        if r.family == "shock_tube":
            assert (wl.ny, wl.nz) == (4, 4) and 256 <= wl.nx <= 2048 and wl.rho.min() == 0.125
        elif r.family == "mach2_blob":
            assert wl.nz == 4 and 256 * 128 <= wl.nx * wl.ny <= 1024 * 256 and wl.faces[0][0] == "eq_inflow"
        else:
            assert 32 <= wl.nx <= 192 and r.tau >= 0.05 - 1e-15


def test_served_tgv_viscosity_reynolds_400():
    """nu = tau theta0 (Sec. II) gives Re = U0 (n / 2 pi) / nu = 400 where the floor does not bind."""
    n, ma = 192, 1.0
    tau = W.tgv_served_tau(n, ma)
    assert abs(ma * W.CS * (n / (2 * np.pi)) / (tau * W.THETA0) - 400.0) < 1e-9
    assert W.tgv_served_tau(32, 0.3) == 0.05
