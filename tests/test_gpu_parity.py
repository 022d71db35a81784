"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the same
seeded inputs.

Tolerances (from the arithmetic): FP64 storage -- fields within 1e-12 relative (rho, theta
pointwise; u relative to max |u|), populations within 1e-12 * w_i * max(1, max|f/w|);
FP32 storage -- 1e-5 relative after 100 steps on a smooth flow.  FP16/BF16 offset storage
errors are reported and only bounded loosely (they are storage-precision limited).
"""

import numpy as np
import pytest

from parity_util import (ensure_built, field_errors, gpu_run, lib_perm, oracle_run, oracle_sampled_step,
                         population_error, site_coords)
from oracle import rd3q81 as O
from paper_2409_05114_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2409_05114_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def perm(B):
    return lib_perm()


@pytest.fixture(scope="module")
def wlib(B):
    return B.lbm_velocities()[1]


def _compare_fp64(wl, steps, tau, perm, wlib, populations=None, tol=1e-12):
    if populations is None:
        f_ref = oracle_run(wl, steps, tau)
    else:
        f_ref = O.run(populations, tau, steps, wl.oracle_bc_x())
    f_gpu, r, u, t = gpu_run(wl, steps, tau, "f64",
                             populations=None if populations is None else populations[:, perm])
    ref_lib = f_ref[:, perm]
    scale = max(1.0, float(np.max(np.abs(ref_lib) / wlib.reshape(1, 81, 1, 1, 1))))
    pe = population_error(ref_lib, f_gpu, wlib)
    assert pe <= tol * scale, (wl.name, pe, scale)
    er = field_errors(O.fields(f_ref), (r, u, t))
    assert max(er) <= tol, (wl.name, er)
    return pe, er


# FP64: the library evaluates the weight polynomials of Table "tab:weights" in FP64 (terms
# ~1e6 cancelling to ~1e4), so its weights carry ~1e-14 relative error against the oracle's
# exact rational ones.  FP32: f~eq evaluated in FP32 (the step kernel's arithmetic); the
# cubic xi-polynomial of the outer shells (|xi|/theta up to ~3) loses a few ulps.
# FP16/BF16: one rounding of d = f/w - 1.
@pytest.mark.parametrize("storage,tol", [("f64", 5e-14), ("f32", 3e-6), ("f16", 2e-3), ("bf16", 1.6e-2)])
def test_init_is_oracle_equilibrium(B, perm, wlib, storage, tol):
    wl = W.smooth_random(13, 6, 5, seed=1, mach=0.5, eta=0.1)
    f_ref = O.init(wl.rho, wl.u, wl.theta)[:, perm]
    f_gpu, r, u, t = gpu_run(wl, 0, 0.1, storage)
    w = wlib.reshape(1, 81, 1, 1, 1)
    err = np.max(np.abs(f_gpu - f_ref) / (w * np.maximum(1.0, np.abs(f_ref / w))))
    assert err <= tol, err


@pytest.mark.parametrize("dims,steps", [((12, 10, 8), 5), ((5, 1, 3), 4), ((33, 3, 2), 3), ((1, 1, 1), 2)])
def test_fp64_periodic_parity(B, perm, wlib, dims, steps):
    wl = W.smooth_random(*dims, seed=3, mach=0.4, eta=0.08)
    _compare_fp64(wl, steps, 0.05, perm, wlib)


def test_fp64_nonequilibrium_state(B, perm, wlib):
    """Arbitrary (non-equilibrium) populations: one step exercises pull + collide fully."""
    wl = W.smooth_random(9, 7, 6, seed=4)
    rng = np.random.default_rng(5)
    f0 = O.init(wl.rho, wl.u, wl.theta) * (1.0 + 0.05 * rng.standard_normal((2, 81, 6, 7, 9)))
    _compare_fp64(wl, 1, 0.2, perm, wlib, populations=f0)
    _compare_fp64(wl, 3, 0.2, perm, wlib, populations=f0)


def test_fp64_sod_zero_gradient(B, perm, wlib):
    wl = W.sod(nx=512, ny=4, nz=4)
    _compare_fp64(wl, 10, wl.paper_tau("lb"), perm, wlib)
    _compare_fp64(wl, 30, wl.paper_tau("literal"), perm, wlib)


def test_fp64_inflow_outflow(B, perm, wlib):
    # Mach-1 blob with vortex: equilibrium inflow at -x, zero-gradient outflow at +x
    wl = W.mach2_blob(nx=96, ny=24, nz=4, mach=1.0)
    _compare_fp64(wl, 4, wl.paper_tau("literal"), perm, wlib)
    # subsonic inflow on +x, zero-gradient on -x (the other orientation)
    wl2 = W.smooth_random(40, 6, 4, seed=6, mach=0.3, eta=0.05,
                          faces=["zero_gradient", ("eq_inflow", 1.05, -0.2, 0.05, 0.0, W.THETA0 * 1.02)])
    _compare_fp64(wl2, 6, 0.1, perm, wlib)


def test_fp64_mach2_blob_first_step(B, perm, wlib):
    """The Mach-2 blob workload itself: after one step some sites already have theta < 0 in
    both codes (outside the series equilibrium's range); parity holds while values are
    finite, and both report the state as unstable."""
    wl = W.mach2_blob(nx=128, ny=32, nz=4)
    tau = wl.paper_tau("lb")
    f_ref = oracle_run(wl, 1, tau)
    assert np.all(np.isfinite(f_ref))
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, "f64", wl.faces)
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_init(ctx, wl.rho.reshape(-1).copy(), wl.u.reshape(-1).copy(), wl.theta.reshape(-1).copy())
        B.lbm_step(ctx, 1)
        f = np.zeros(2 * 81 * wl.nx * wl.ny * wl.nz)
        B.lbm_get_populations(ctx, f)
        unstable = False
        try:
            B.lbm_sync(ctx)
        except B.LbmUnstable:
            unstable = True
    finally:
        B.lbm_destroy(ctx)
    ref = f_ref[:, perm]
    # Where theta is near 0 the equilibrium (1/theta^3 terms) amplifies rounding: compare
    # element-wise relative to each value.
    np.testing.assert_allclose(f.reshape(ref.shape), ref, rtol=1e-9, atol=1e-13)
    _, _, th = O.fields(f_ref)
    assert unstable == bool((th <= 0).any())


def test_fp64_taylor_green(B, perm, wlib):
    wl = W.taylor_green(16)
    _compare_fp64(wl, 20, wl.paper_tau("lb"), perm, wlib)


@pytest.mark.parametrize("fp64_moments", [False, True])
def test_fp32_taylor_green_100_steps(B, perm, wlib, fp64_moments):
    """Smooth compressible TGV, Ma 0.5, 32^3, 100 steps: FP32 storage within 1e-5 of FP64."""
    wl = W.taylor_green(32)
    tau = wl.paper_tau("lb")
    ref = O.fields(oracle_run(wl, 100, tau))
    _, r, u, t = gpu_run(wl, 100, tau, "f32", fp64_moments=fp64_moments)
    er = field_errors(ref, (r, u, t))
    print("fp32 TGV32 100 steps, fp64_moments=%s: rel err rho %.3g u %.3g theta %.3g" % (fp64_moments, *er))
    assert max(er) <= 1e-5, er


# Bounds about 3x the measured errors (FP32 2.6e-7 / 5.1e-7 / 2.1e-7 in rho / u / theta; FP16
# offsets 2.6e-4 / 5.3e-4 / 2.2e-4; BF16 offsets 2.2e-3 / 4.7e-3 / 1.8e-3): the storage rounding of
# d = f/w - 1 sets them, so a regression of the arithmetic shows well inside a storage-sized bound.
@pytest.mark.parametrize("fp64_moments", [True, False])
@pytest.mark.parametrize("storage,bound", [("f32", 1e-5), ("f16", 2e-3), ("bf16", 1.5e-2)])
def test_storage_precision_errors_hit(B, storage, bound, fp64_moments):
    """Decaying turbulence (HIT generator), 16^3, 20 steps: error of each storage precision
    against the FP64 oracle, with FP64-quality moment sums and with FP32 ones (for FP16/BF16 on
    this even grid the two-sites-per-thread kernel)."""
    wl = W.hit(16, seed=2409)
    tau = wl.paper_tau("lb")
    ref = O.fields(oracle_run(wl, 20, tau))
    _, r, u, t = gpu_run(wl, 20, tau, storage, fp64_moments=fp64_moments)
    er = field_errors(ref, (r, u, t))
    print("%s HIT16 20 steps, fp64_moments=%s: rel err rho %.3g u %.3g theta %.3g" % (storage, fp64_moments, *er))
    assert all(np.isfinite(er)) and max(er) <= bound, er


def test_conservation_on_device(B):
    """Sum rho, rho u and <f, c^2> over a periodic grid are conserved by ten steps: FP64 to
    round-off; FP32 storage to the rounding of the stored values (the step's f~eq-shaped
    conservation projection removes the FP32 defects of each update).  lbm_totals sums the
    stored values in FP64."""
    wl = W.smooth_random(20, 12, 10, seed=8, mach=0.5, eta=0.1)
    for storage, tol in (("f64", 1e-13), ("f32", 2e-7)):
        cfg = B.make_config(wl.nx, wl.ny, wl.nz, 0.05, storage)
        ctx = B.lbm_create(cfg)
        try:
            B.lbm_init(ctx, wl.rho.reshape(-1).copy(), wl.u.reshape(-1).copy(), wl.theta.reshape(-1).copy())
            t0 = B.lbm_totals(ctx)
            B.lbm_step(ctx, 10)
            t1 = B.lbm_totals(ctx)
            again = B.lbm_totals(ctx)
        finally:
            B.lbm_destroy(ctx)
        np.testing.assert_array_equal(t1, again)           # deterministic reduction
        scale = np.array([t0[0]] * 4 + [t0[4]])
        print(storage, "drift / scale", (t1 - t0) / scale)
        assert np.all(np.abs(t1 - t0) <= tol * scale), (storage, t1 - t0)
        ref = O.totals(O.init(wl.rho, wl.u, wl.theta))
        assert np.all(np.abs(t0 - ref) <= max(tol, 1e-13) * scale)


def test_unstable_flag_reported(B):
    """Strong Sod under the tau_lb reading leaves the series equilibrium's range within ~20
    steps: the run must report LBM_EUNSTABLE (host-side detection; nothing faults)."""
    wl = W.sod(nx=512, ny=4, nz=4)
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, wl.paper_tau("lb"), "f32", wl.faces)
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_init(ctx, wl.rho.reshape(-1).copy(), wl.u.reshape(-1).copy(), wl.theta.reshape(-1).copy())
        B.lbm_step(ctx, 60)
        with pytest.raises(B.LbmUnstable):
            B.lbm_sync(ctx)
        S = wl.sites
        with pytest.raises(B.LbmUnstable):
            B.lbm_moments(ctx, np.zeros(S), np.zeros(3 * S), np.zeros(S))
        # a fresh init clears the flag
        B.lbm_init(ctx, wl.rho.reshape(-1).copy(), wl.u.reshape(-1).copy(), wl.theta.reshape(-1).copy())
        B.lbm_step(ctx, 2)
        B.lbm_sync(ctx)
    finally:
        B.lbm_destroy(ctx)


def test_api_edge_cases(B):
    wl = W.smooth_random(8, 4, 4, seed=9)
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, 0.1, "f32")
    ctx = B.lbm_create(cfg)
    try:
        with pytest.raises(B.LbmError) as ei:
            B.lbm_step(ctx, 1)                              # before init
        assert ei.value.status == B.LBM_EINVAL
        B.lbm_init(ctx, wl.rho.reshape(-1).copy(), wl.u.reshape(-1).copy(), wl.theta.reshape(-1).copy())
        f0 = np.zeros(2 * 81 * wl.nx * wl.ny * wl.nz)
        B.lbm_get_populations(ctx, f0)
        B.lbm_step(ctx, 0)                                  # no-op
        f1 = np.zeros_like(f0)
        B.lbm_get_populations(ctx, f1)
        np.testing.assert_array_equal(f0, f1)
        with pytest.raises(B.LbmError):
            B.lbm_step(ctx, -1)
        with pytest.raises(B.LbmError):
            B.lbm_probe(ctx, [wl.sites])                    # out of range
        p = B.lbm_probe(ctx, [0, wl.sites - 1])
        ff = f1.reshape(2, 81, -1)
        np.testing.assert_array_equal(p[0], ff[0, :, 0])
        np.testing.assert_array_equal(p[1], ff[1, :, -1])
        # set/get round trip is exact for FP32-representable values
        B.lbm_set_populations(ctx, f1)
        f2 = np.zeros_like(f1)
        B.lbm_get_populations(ctx, f2)
        np.testing.assert_array_equal(f1, f2)
        assert B.lbm_launch_count(ctx) > 0
    finally:
        B.lbm_destroy(ctx)


def test_device_pointer_path_matches_host(B):
    import torch
    wl = W.smooth_random(16, 8, 4, seed=10)
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, 0.1, "f32", stream=torch.cuda.current_stream())
    ctx = B.lbm_create(cfg)
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
        B.lbm_init(ctx, dev(wl.rho), dev(wl.u), dev(wl.theta))
        B.lbm_step(ctx, 3)
        S = wl.sites
        r, u, t = (torch.zeros(k * S, dtype=torch.float64, device="cuda") for k in (1, 3, 1))
        B.lbm_moments(ctx, r, u, t)
        rh, uh, th = np.zeros(S), np.zeros(3 * S), np.zeros(S)
        B.lbm_moments(ctx, rh, uh, th)
        np.testing.assert_array_equal(r.cpu().numpy(), rh)
        np.testing.assert_array_equal(u.cpu().numpy(), uh)
        np.testing.assert_array_equal(t.cpu().numpy(), th)
    finally:
        B.lbm_destroy(ctx)


def _round_f16_offsets(f):
    """The values FP16 offset storage holds for populations f [81, ...] (oracle order):
    w (1 + d) with d = f / w - 1 rounded to FP16."""
    w = O.velocity_set().w.reshape((81,) + (1,) * (f.ndim - 1))
    return w * (1.0 + (f / w - 1.0).astype(np.float16).astype(np.float64))


def _sampled_full_size(B, perm, wlib, wl, storage, tol, nsamples=96, eq="series", collision="bgk",
                       fp64_moments=False):
    tau = wl.paper_tau("lb")
    rng = np.random.default_rng(123)
    n = wl.nx * wl.ny * wl.nz
    # random sites plus the corners and faces of both sublattices (wrap-around paths)
    edge = [0, wl.nx - 1, n - 1, n - wl.nx, n, 2 * n - 1, n + wl.nx * wl.ny - 1]
    sites = np.unique(np.concatenate([rng.integers(0, 2 * n, nsamples), edge]))
    store = _round_f16_offsets if storage == "f16" else None
    ref = oracle_sampled_step(wl, sites, tau, eq=eq, collision=collision, store=store)[perm].T  # [K, 81]
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, storage, fp64_moments=fp64_moments, equilibrium=eq,
                        collision=collision)
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_init(ctx, wl.rho.reshape(-1), wl.u.reshape(-1), wl.theta.reshape(-1))
        B.lbm_step(ctx, 1)
        got = B.lbm_probe(ctx, sites)
    finally:
        B.lbm_destroy(ctx)
    err = np.max(np.abs(got - ref) / (wlib * np.maximum(1.0, np.abs(ref / wlib))))
    print("%s %s %s/%s%s sampled 1-step population error %.3g" %
          (wl.name, storage, eq, collision, " fp64 moments" if fp64_moments else "", err))
    assert err <= tol, err


@pytest.fixture(scope="module")
def tgv512():
    return W.taylor_green(512)


# FP32 per-population bound for one step from FP32 inputs: the FP32 evaluation of the
# cubic xi-polynomial of the outer shells (emulated bound 1.3e-5), times 3.
@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 4e-5)])
def test_full_size_tgv128_sampled(B, perm, wlib, storage, tol):
    _sampled_full_size(B, perm, wlib, W.taylor_green(128), storage, tol)


def test_full_size_tgv512_fp32_sampled(B, perm, wlib, tgv512):
    """The roofline point of the benchmark: 512^3 TGV, FP32 storage (2 x 87 GB)."""
    _sampled_full_size(B, perm, wlib, tgv512, "f32", 4e-5, nsamples=64)


def test_full_size_tgv512_fp32_fp64_moments_sampled(B, perm, wlib, tgv512):
    """512^3 TGV, FP32 storage with FP64-quality moments (exact integer sums), as the bench
    times it."""
    _sampled_full_size(B, perm, wlib, tgv512, "f32", 4e-5, nsamples=64, fp64_moments=True)


def test_full_size_tgv512_fp16_sampled(B, perm, wlib, tgv512):
    """512^3 TGV, FP16 offsets: the two-sites-per-thread kernel as the bench times it.  The
    oracle steps the FP16-rounded initial state; the kernel's FP32 arithmetic and its rounding of
    the result to FP16 leave at most about one FP16 unit of the offset (4.9e-4 below |d| = 1);
    measured 4.3e-4."""
    _sampled_full_size(B, perm, wlib, tgv512, "f16", 1.3e-3, nsamples=64)


@pytest.mark.parametrize("collision", ["bgk", "entropic"])
def test_full_size_tgv256_entropic_sampled(B, perm, wlib, collision):
    """256^3 TGV, FP32 storage, exact entropic equilibrium with BGK or with the entropic alpha
    (the kernels of the served mix and the entropic-alpha bench line), sampled one step.  The FP32
    Newton for the multipliers stops at 1e-6 of the moments; measured 1.9e-5 (BGK) and 1.8e-5
    (entropic alpha)."""
    _sampled_full_size(B, perm, wlib, W.taylor_green(256), "f32", 6e-5, nsamples=64, eq="entropic",
                       collision=collision)
