"""Continuous-batching server (lbm_server_*): each case's result is bitwise the same served
alone and in a mix (one kernel per kind of case, independent sites) and agrees with the
single-case API within the storage precision's tolerance, for the series and the exact entropic
equilibrium (a Mach-2 blob, a strong Sod tube and a Mach-1 Taylor-Green vortex among them);
served results match the FP64 oracle,
admission respects the HBM budget, an unstable case is retired early without disturbing
the others, and waits are bounded.  Failures are made on the host (a state outside the
equilibrium's range, an over-budget request, a short timeout); nothing faults the GPU."""

import numpy as np
import pytest

from parity_util import ensure_built, field_errors, oracle_run
from oracle import rd3q81 as O
from paper_2409_05114_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2409_05114_gb300 import binding
    return binding


def _fields(wl):
    return (np.ascontiguousarray(wl.rho, dtype=np.float64).reshape(-1),
            np.ascontiguousarray(wl.u, dtype=np.float64).reshape(-1),
            np.ascontiguousarray(wl.theta, dtype=np.float64).reshape(-1))


def _single(B, wl, storage, tau, nsteps, eq="series"):
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, storage, wl.faces, equilibrium=eq)
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_init(ctx, *_fields(wl))
        B.lbm_step(ctx, nsteps)
        S = wl.sites
        out = (np.zeros(S), np.zeros(3 * S), np.zeros(S))
        try:
            B.lbm_moments(ctx, *out)
            status = B.LBM_OK
        except B.LbmUnstable:
            status = B.LBM_EUNSTABLE
    finally:
        B.lbm_destroy(ctx)
    return status, out


def _serve(B, items, budget=8 << 30, max_cases=16, timeout=300.0):
    """items: (workload, storage, tau, steps[, equilibrium])."""
    srv = B.lbm_server_create(budget, max_cases)
    try:
        tickets = []
        for it in items:
            wl, storage, tau, n = it[:4]
            eq = it[4] if len(it) > 4 else "series"
            cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, storage, wl.faces, equilibrium=eq)
            tickets.append(B.lbm_submit(srv, cfg, *_fields(wl), n))
        results = []
        for it, t in zip(items, tickets):
            wl = it[0]
            assert B.lbm_wait(srv, t, timeout) == B.LBM_OK
            S = wl.sites
            out = (np.zeros(S), np.zeros(3 * S), np.zeros(S))
            st, lat = B.lbm_poll(srv, t, *out)
            assert lat > 0.0
            results.append((st, out))
        stats = B.lbm_server_get_stats(srv)
    finally:
        B.lbm_server_destroy(srv)
    return results, stats


def _items():
    return [
        (W.taylor_green(16, mach=0.5), "f32", W.paper_tau(0.51, "lb"), 30),
        (W.taylor_green(24, mach=0.7), "f16", W.paper_tau(0.51, "lb"), 20),
        (W.sod(nx=256, ny=4, nz=4), "f32", W.paper_tau(0.6, "literal"), 40),
        (W.mach2_blob(64, 32, 4, mach=0.5, vortex=0.1), "f16", W.paper_tau(0.55, "literal"), 25),
        (W.smooth_random(33, 5, 4, seed=3, mach=0.3), "bf16", 0.1, 15),
        # exact entropic equilibrium (Sec. III): the config-5 families in their Mach range
        (W.mach2_blob(64, 16, 4), "f32", W.paper_tau(0.55, "lb"), 30, "entropic"),
        (W.mach2_blob(64, 16, 4), "f16", W.paper_tau(0.55, "lb"), 30, "entropic"),
        (W.sod(nx=128, ny=4, nz=4), "f32", W.paper_tau(0.6, "lb"), 40, "entropic"),
        (W.taylor_green(16, mach=1.0), "bf16", W.paper_tau(0.55, "lb"), 20, "entropic"),
    ]


# Served vs the single-case kernel: the same arithmetic compiled in two kernels (FP32
# contraction may differ by an ulp per step); bounded like the FP32 parity tests, and like the
# storage-precision tests for FP16/BF16.
_SERVED_VS_SINGLE_TOL = {"f32": 1e-5, "f16": 2e-3, "bf16": 1e-2}


def _rel(a, b, S):
    r0, u0, t0 = a
    r1, u1, t1 = b
    return max(np.max(np.abs(r1 - r0) / np.abs(r0)), np.max(np.abs(u1 - u0)) / max(np.max(np.abs(u0)), 1e-30),
               np.max(np.abs(t1 - t0) / np.abs(t0)))


def test_results_identical_alone_and_in_mix(B):
    items = _items()
    mixed, stats = _serve(B, items)
    assert stats["completed"] == len(items) and stats["unstable"] == 0
    assert stats["graph_launches"] > 0
    # each case served alone gives bitwise the same result as in the mix
    for item, (s1, b) in zip(items, mixed):
        assert s1 == B.LBM_OK
        (s0, a), = _serve(B, [item])[0]
        assert s0 == B.LBM_OK
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    # and agrees with the single-case API within the storage's tolerance
    for it, (_, b) in zip(items, mixed):
        wl, st, tau, n = it[:4]
        eq = it[4] if len(it) > 4 else "series"
        s0, a = _single(B, wl, st, tau, n, eq)
        assert s0 == B.LBM_OK
        assert _rel(a, b, wl.sites) <= _SERVED_VS_SINGLE_TOL[st], (wl.name, st, eq)


def test_served_case_matches_oracle(B):
    wl = W.taylor_green(12, mach=0.5)
    tau = W.paper_tau(0.51, "lb")
    (st, (r, u, t)), = _serve(B, [(wl, "f32", tau, 30)])[0]
    assert st == B.LBM_OK
    shp = (2, wl.nz, wl.ny, wl.nx)
    ref = O.fields(oracle_run(wl, 30, tau))
    er = field_errors(ref, (r.reshape(shp), u.reshape((3,) + shp), t.reshape(shp)))
    assert max(er) <= 1e-5, er


def test_served_entropic_mach2_matches_oracle(B):
    """A served Mach-2 blob with the exact entropic equilibrium (Sec. III), FP32 storage, against
    the FP64 oracle with the same equilibrium: within the FP32 bound of the single-case tests."""
    wl = W.mach2_blob(32, 16, 4)
    tau = W.paper_tau(0.55, "lb")
    (st, (r, u, t)), = _serve(B, [(wl, "f32", tau, 10, "entropic")])[0]
    assert st == B.LBM_OK
    shp = (2, wl.nz, wl.ny, wl.nx)
    ref = O.fields(oracle_run(wl, 10, tau, eq="entropic"))
    er = field_errors(ref, (r.reshape(shp), u.reshape((3,) + shp), t.reshape(shp)))
    print("served entropic f32 Mach-2 blob 10 steps: rel err rho %.3g u %.3g theta %.3g" % er)
    assert max(er) <= 1e-5, er


def test_admission_respects_budget(B):
    wl = W.taylor_green(32)
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, 0.01, "f32")
    # a served case holds two population buffers; lbm_footprint adds a context's scratch and
    # staging to those, so it bounds one case's footprint from above (the library pads rows to
    # whole x tiles, so the buffers are not 81 x sites x 4 bytes exactly)
    one = B.lbm_footprint(cfg)
    items = [(wl, "f32", 0.01, 10)] * 3
    results, stats = _serve(B, items, budget=int(one * 1.5))
    assert all(st == B.LBM_OK for st, _ in results)
    assert stats["peak_resident_bytes"] <= int(one * 1.5)
    assert stats["admitted"] == 3
    # a case that alone exceeds the budget is refused at submission
    srv = B.lbm_server_create(one // 2, 4)
    try:
        with pytest.raises(B.LbmError) as ei:
            B.lbm_submit(srv, cfg, *_fields(wl), 10)
        assert ei.value.status == B.LBM_ENOMEM
        bad = B.make_config(wl.nx, wl.ny, wl.nz, 0.01, "f64")
        with pytest.raises(B.LbmError) as ei:
            B.lbm_submit(srv, bad, *_fields(wl), 10)
        assert ei.value.status == B.LBM_EINVAL
        assert B.lbm_poll(srv, 12345)[0] == B.LBM_ENOTFOUND
    finally:
        B.lbm_server_destroy(srv)


def test_first_fit_admission_lets_small_cases_pass(B):
    """When the oldest waiting request does not fit the free budget, a later one that fits is
    admitted ahead of it: with room for one large case and two small ones, the small cases
    submitted after a second large one finish before it."""
    big, small = W.taylor_green(48), W.taylor_green(16)
    tau = W.paper_tau(0.55, "lb")
    one_big = B.lbm_footprint(B.make_config(48, 48, 48, tau, "f32"))
    one_small = B.lbm_footprint(B.make_config(16, 16, 16, tau, "f32"))
    items = [(big, "f32", tau, 2000), (big, "f32", tau, 50), (small, "f32", tau, 20), (small, "f32", tau, 20)]
    srv = B.lbm_server_create(one_big + 2 * one_small, 8)
    try:
        tickets = [B.lbm_submit(srv, B.make_config(w.nx, w.ny, w.nz, t, st), *_fields(w), n)
                   for w, st, t, n in items]
        lat = []
        for t in tickets:
            assert B.lbm_wait(srv, t, 300.0) == B.LBM_OK
            st, l = B.lbm_poll(srv, t)
            assert st == B.LBM_OK
            lat.append(l)
        stats = B.lbm_server_get_stats(srv)
    finally:
        B.lbm_server_destroy(srv)
    assert lat[2] < lat[0] and lat[3] < lat[0]      # the small cases ran beside the first large one
    assert lat[2] < lat[1] and lat[3] < lat[1]      # ... ahead of the second
    assert stats["peak_resident_bytes"] <= one_big + 2 * one_small


def test_unstable_case_retired_early_others_unaffected(B):
    unstable = (W.sod(nx=512, ny=4, nz=4), "f32", W.paper_tau(0.6, "lb"), 100000)
    good = _items()[0]
    (_, alone), = _serve(B, [good])[0]
    results, stats = _serve(B, [unstable, good], timeout=120.0)
    assert results[0][0] == B.LBM_EUNSTABLE
    assert results[1][0] == B.LBM_OK
    assert stats["unstable"] == 1
    for x, y in zip(alone, results[1][1]):
        np.testing.assert_array_equal(x, y)


def test_bounded_wait_times_out(B):
    wl = W.taylor_green(64)
    srv = B.lbm_server_create(4 << 30, 4)
    try:
        cfg = B.make_config(wl.nx, wl.ny, wl.nz, 0.01, "f32")
        t = B.lbm_submit(srv, cfg, *_fields(wl), 200000)
        assert B.lbm_wait(srv, t, 0.05) == B.LBM_ETIMEOUT
        assert B.lbm_poll(srv, t)[0] == B.LBM_EBUSY
    finally:
        B.lbm_server_destroy(srv)                           # drops the running case
