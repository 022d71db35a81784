"""Bounce-back walls on the GPU (LBM_BC_BOUNCE_BACK) against the FP64 oracle, whose wall is pinned
in tests/test_oracle_bounce_back.py: a shock tube set up like the paper's Sod case (walls at both
x ends, periodic y and z) run until its waves have reflected from the walls, one wall with another
face kind, FP64 to 1e-12 and FP32 to its storage precision; AA streaming and the fused host-field
call against ping-pong; a closed box conserves mass and energy on the device.  The tube's jump is
rho 1 | 0.5, theta theta0 | 0.9 theta0: with the full Sod jump (1 | 0.125) on a tube this short the
series equilibrium breaks down (rho and theta negative at step 19) in the oracle too, walls or not."""

import numpy as np
import pytest

from parity_util import ensure_built, field_errors, gpu_run, lib_perm, oracle_run, population_error
from oracle import rd3q81 as O
from paper_2409_05114_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2409_05114_gb300 import binding
    return binding


def _cases():
    sod = W.shock_tube(nx=40, ny=3, nz=2, rho_right=0.5, theta_right=0.9, walls=True)  # walls hit by step 20
    mixed = W.smooth_random(24, 4, 3, seed=7, mach=0.3, faces=["bounce_back", "zero_gradient"])
    inflow = W.smooth_random(20, 3, 2, seed=8, mach=0.2,
                             faces=[("eq_inflow", 1.0, 0.1 * W.CS, 0.0, 0.0, W.THETA0), "bounce_back"])
    return [sod, mixed, inflow]


@pytest.mark.parametrize("k", [0, 1, 2])
def test_fp64_parity(B, k):
    wl = _cases()[k]
    tau = wl.paper_tau("lb")
    steps = 30
    f_ref = oracle_run(wl, steps, tau)
    perm = lib_perm()
    w = B.lbm_velocities()[1]
    f_gpu, r, u, t = gpu_run(wl, steps, tau, "f64")
    ref = f_ref[:, perm]
    scale = max(1.0, float(np.max(np.abs(ref) / w.reshape(1, 81, 1, 1, 1))))
    assert population_error(ref, f_gpu, w) <= 1e-12 * scale
    assert max(field_errors(O.fields(f_ref), (r, u, t))) <= 1e-12


def test_fp32_sod_walls(B):
    wl = _cases()[0]
    tau = wl.paper_tau("lb")
    ref = O.fields(oracle_run(wl, 30, tau))
    _, r, u, t = gpu_run(wl, 30, tau, "f32")
    er = field_errors(ref, (r, u, t))
    assert max(er) <= 2e-5, er


def _fields(wl):
    return (np.ascontiguousarray(wl.rho).reshape(-1), np.ascontiguousarray(wl.u).reshape(-1),
            np.ascontiguousarray(wl.theta).reshape(-1))


def _moments_after(B, wl, storage, streaming, steps):
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, wl.paper_tau(), storage, wl.faces, streaming=streaming)
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_init(ctx, *_fields(wl))
        out = []
        for n in steps:
            B.lbm_step(ctx, n)
            S = wl.sites
            r, u, t = np.zeros(S), np.zeros(3 * S), np.zeros(S)
            B.lbm_moments(ctx, r, u, t)
            out.append((r, u, t, B.lbm_totals(ctx)))
        return out
    finally:
        B.lbm_destroy(ctx)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 1e-6)])
def test_aa_matches_pingpong(B, storage, tol):
    for wl in _cases():
        steps = [1, 1, 3, 12]                       # both AA layouts, then graph replay
        a = _moments_after(B, wl, storage, "aa", steps)
        p = _moments_after(B, wl, storage, "pingpong", steps)
        for x, y in zip(a, p):
            for g, h in zip(x, y):
                assert np.max(np.abs(g - h)) <= tol * max(1.0, np.max(np.abs(h)))


def test_closed_box_conserves_on_device(B):
    wl = W.smooth_random(32, 8, 6, seed=3, mach=0.4, faces=["bounce_back", "bounce_back"])
    for streaming in ("pingpong", "aa"):
        out = _moments_after(B, wl, "f64", streaming, [0, 10, 25])
        t0 = out[0][3]
        for *_, t in out[1:]:
            assert abs(t[0] - t0[0]) <= 1e-12 * abs(t0[0])
            assert abs(t[4] - t0[4]) <= 1e-12 * abs(t0[4])


@pytest.mark.parametrize("streaming", ["pingpong", "aa"])
@pytest.mark.parametrize("shape", [(64, 2048, 20), (32, 32768, 10)])
def test_fused_call_with_walls(B, shape, streaming):
    """Several slabs (8 planes) and slabs one plane thick, walls on both x faces: the fused call
    equals the separate calls bitwise."""
    torch = pytest.importorskip("torch")
    nx, ny, nz = shape
    wl = W.smooth_random(nx, ny, nz, seed=nz, mach=0.3, faces=["bounce_back", "bounce_back"])
    fields = _fields(wl)
    cfg = B.make_config(nx, ny, nz, wl.paper_tau(), "f32", wl.faces, streaming=streaming)
    S = wl.sites
    for n in (1, 2, 3):
        ctx = B.lbm_create(cfg)
        try:
            B.lbm_init(ctx, *fields)
            B.lbm_step(ctx, n)
            ref = [np.zeros(S), np.zeros(3 * S), np.zeros(S)]
            B.lbm_moments(ctx, *ref)
        finally:
            B.lbm_destroy(ctx)
        pin_in = [torch.from_numpy(a.copy()).pin_memory() for a in fields]
        pin_out = [torch.zeros(a.size, dtype=torch.float64).pin_memory() for a in fields]
        ctx = B.lbm_create(cfg)
        try:
            B.lbm_advance_fields(ctx, *[t.numpy() for t in pin_in], n, *[t.numpy() for t in pin_out])
        finally:
            B.lbm_destroy(ctx)
        for g, h in zip(pin_out, ref):
            np.testing.assert_array_equal(g.numpy(), h)


def test_served_cases_reject_walls(B):
    srv = B.lbm_server_create(1 << 30, 4)
    try:
        wl = W.sod(nx=32, ny=2, nz=2, walls=True)
        cfg = B.make_config(wl.nx, wl.ny, wl.nz, 0.1, "f32", wl.faces)
        with pytest.raises(B.LbmError):
            B.lbm_submit(srv, cfg, *_fields(wl), 10)
    finally:
        B.lbm_server_destroy(srv)
