"""GPU parity of the series equilibrium with the exact temperature weights W(theta) of App. B,
Eq. (zeroveleq) (config equilibrium = LBM_EQ_SERIES_EXACT_W), against the oracle.

Tolerances: FP64 -- both sides solve the 1-D relation theta'(G) to round-off, so populations
within 1e-11 of the weights; FP32 -- fields within 1e-5 after 20 steps, as for the series
weights."""

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


@pytest.fixture(scope="module")
def perm(B):
    return lib_perm()


@pytest.fixture(scope="module")
def wlib(B):
    return B.lbm_velocities()[1]


@pytest.mark.parametrize("dims,steps,mach,eta", [((10, 8, 6), 0, 0.5, 0.4), ((10, 8, 6), 4, 0.5, 0.3),
                                                  ((13, 3, 2), 3, 0.9, 0.15)])
def test_fp64_exact_w_parity(B, perm, wlib, dims, steps, mach, eta):
    wl = W.smooth_random(*dims, seed=31, mach=mach, eta=eta)
    tau = 0.1
    f_or = oracle_run(wl, steps, tau, eq="series_exact_w")
    f, r, u, t = gpu_run(wl, steps, tau, "f64", eq="series_exact_w", check_stable=True)
    err = population_error(f_or[:, perm], f, wlib)
    print("exact-W f64 %s %d steps: population error %.3g" % (dims, steps, err))
    assert err <= 1e-11
    er = field_errors(O.fields(f_or), (r, u, t))
    assert max(er) <= 1e-11, er


def test_exact_weights_differ_from_series_when_hot(B):
    wl = W.smooth_random(10, 8, 6, seed=31, mach=0.3, eta=0.4)
    f1, _, _, _ = gpu_run(wl, 0, 0.1, "f64", eq="series_exact_w")
    f2, _, _, _ = gpu_run(wl, 0, 0.1, "f64", eq="series")
    assert np.max(np.abs(f1 - f2)) > 1e-6 * np.max(np.abs(f2))


@pytest.mark.parametrize("wl_name,steps", [("tgv16", 20), ("hot_random", 10)])
def test_exact_w_f32(B, wl_name, steps):
    if wl_name == "tgv16":
        wl = W.taylor_green(16, mach=0.5)
        tau = wl.paper_tau("lb")
    else:
        wl = W.smooth_random(16, 8, 6, seed=41, mach=0.5, eta=0.35)
        tau = 0.1
    ref = O.fields(oracle_run(wl, steps, tau, eq="series_exact_w"))
    _, r, u, t = gpu_run(wl, steps, tau, "f32", eq="series_exact_w", check_stable=True)
    er = field_errors(ref, (r, u, t))
    print("exact-W f32 %s %d steps: rel err rho %.3g u %.3g theta %.3g" % (wl_name, steps, *er))
    assert max(er) <= 1e-5, er
