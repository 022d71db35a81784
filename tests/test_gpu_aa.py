"""In-place (AA) streaming against ping-pong: one population buffer, the two AA step kinds
alternating, every boundary kind.  The arithmetic of a site update is the same, only the
addresses differ; the step kinds are separately compiled kernels, so a multiply-add may be
contracted differently and results agree to rounding (FP64 1e-13, FP32 1e-6, FP16 offsets one
storage rounding), while any misplaced population would show at O(1).  Checked after any number
of steps: odd counts end in the pushed layout, even counts in the own layout, and 12 steps take
the captured-graph path."""

import numpy as np
import pytest

from parity_util import ensure_built
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


def _run(B, wl, tau, storage, steps, streaming, eq="series", collision="bgk", fp64_moments=False):
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, storage, wl.faces, equilibrium=eq, collision=collision,
                        streaming=streaming, fp64_moments=fp64_moments)
    ctx = B.lbm_create(cfg)
    out = []
    try:
        B.lbm_init(ctx, *_fields(wl))
        for n in steps:
            B.lbm_step(ctx, n)
            S = wl.sites
            r, u, t = np.zeros(S), np.zeros(3 * S), np.zeros(S)
            B.lbm_moments(ctx, r, u, t)
            f = np.zeros(S * 81)
            B.lbm_get_populations(ctx, f)
            tot = B.lbm_totals(ctx)
            pr = B.lbm_probe(ctx, np.array([0, S // 3, S - 1], dtype=np.int64))
            out.append((r, u, t, f, tot, pr))
    finally:
        B.lbm_destroy(ctx)
    return out


_TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-3, "bf16": 1.6e-2}


def _same(a, b, storage):
    for x, y in zip(a, b):
        for p, q in zip(x, y):
            scale = max(float(np.max(np.abs(q))), 1e-300)
            assert float(np.max(np.abs(p - q))) <= _TOL[storage] * scale


# Odd nx: ping-pong then runs the one-site-per-thread kernel whose arithmetic the AA kernels
# share (with nx even, FP16/BF16 ping-pong runs the two-sites-per-thread kernel, which rounds
# differently and is compared with the oracle in test_gpu_pair.py).
CASES = [
    ("tgv", lambda: W.taylor_green(13, mach=0.5), "lb"),
    ("sod", lambda: W.sod(nx=63, ny=4, nz=3), "lb"),
    ("blob", lambda: W.mach2_blob(39, 8, 4, mach=0.5, vortex=0.1), "literal"),
]


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("name,make,reading", CASES)
def test_aa_matches_pingpong(B, storage, name, make, reading):
    wl = make()
    tau = wl.paper_tau(reading)
    steps = [0, 1, 1, 3, 12]              # cumulative 0, 1, 2, 5, 17: both layouts, graph replay
    _same(_run(B, wl, tau, storage, steps, "aa"), _run(B, wl, tau, storage, steps, "pingpong"), storage)


@pytest.mark.parametrize("eq,collision", [("entropic", "bgk"), ("entropic", "entropic"), ("series_exact_w", "bgk")])
def test_aa_other_equilibria(B, eq, collision):
    wl = W.mach2_blob(32, 8, 4, mach=0.5, vortex=0.1)
    tau = wl.paper_tau("literal")
    steps = [1, 2, 12]
    _same(_run(B, wl, tau, "f32", steps, "aa", eq, collision), _run(B, wl, tau, "f32", steps, "pingpong", eq, collision),
          "f32")


def test_aa_set_get_roundtrip_and_footprint(B):
    wl = W.smooth_random(9, 7, 5, seed=3, mach=0.4, faces=["zero_gradient", "zero_gradient"])
    cfg_aa = B.make_config(wl.nx, wl.ny, wl.nz, 0.1, "f64", wl.faces, streaming="aa")
    cfg_pp = B.make_config(wl.nx, wl.ny, wl.nz, 0.1, "f64", wl.faces)
    one = 2 * 81 * wl.nx * wl.ny * wl.nz * 8
    assert B.lbm_footprint(cfg_pp) - B.lbm_footprint(cfg_aa) >= one
    # a state near equilibrium: the initial populations, perturbed by 1 %
    ctx = B.lbm_create(cfg_pp)
    try:
        B.lbm_init(ctx, *_fields(wl))
        f0 = np.zeros(wl.sites * 81)
        B.lbm_get_populations(ctx, f0)
    finally:
        B.lbm_destroy(ctx)
    f0 *= 1.0 + 0.01 * np.random.default_rng(1).uniform(-1, 1, f0.size)
    res = []
    for cfg in (cfg_aa, cfg_pp):
        ctx = B.lbm_create(cfg)
        try:
            B.lbm_set_populations(ctx, f0)
            g = np.zeros_like(f0)
            B.lbm_get_populations(ctx, g)
            np.testing.assert_array_equal(g, f0)
            B.lbm_step(ctx, 3)
            B.lbm_get_populations(ctx, g)
            res.append(g.copy())
        finally:
            B.lbm_destroy(ctx)
    assert np.max(np.abs(res[0] - res[1])) <= 1e-13 * np.max(np.abs(res[1]))


def test_aa_diagnostics(B):
    wl = W.taylor_green(10, mach=0.5)
    vals = []
    for st in ("aa", "pingpong"):
        ctx = B.lbm_create(B.make_config(wl.nx, wl.ny, wl.nz, wl.paper_tau("lb"), "f32", wl.faces, streaming=st))
        try:
            B.lbm_init(ctx, *_fields(wl))
            B.lbm_step(ctx, 3)
            vals.append(B.lbm_diagnostics(ctx))
        finally:
            B.lbm_destroy(ctx)
    np.testing.assert_allclose(vals[0], vals[1], rtol=1e-6)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_aa_fp64_moments_matches_pingpong(B, storage):
    """FP64-quality moment sums (double words) with in-place streaming, against ping-pong with the
    same option, over every boundary kind's case."""
    for name, make, reading in CASES:
        wl = make()
        tau = wl.paper_tau(reading)
        steps = [1, 2, 12]
        a = _run(B, wl, tau, storage, steps, "aa", fp64_moments=True)
        b = _run(B, wl, tau, storage, steps, "pingpong", fp64_moments=True)
        _same(a, b, storage)
