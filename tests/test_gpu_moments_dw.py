"""The moment read-back of FP32 / FP16 storage (lbm_moments: FP32 shell sums, then double-word
arithmetic) against FP64 sums of the very values the library stores.  The populations are chosen
so that every FP32 shell sum is exact -- per shell, integers below 2^18 times one power of two --
which leaves only the double-word combination, reciprocal and products: rho, u and theta must
agree with the FP64 definition (Eq. (conslaws)) to ~1e-13, far below the 6e-8 an FP32
combination would give.  FP16 offsets (d = f / w - 1, dyadic, exact in FP16) check the offset
path, whose weighted offset sums round once in FP32 (relative 1e-7 of a ~1e-2 deviation)."""

import numpy as np
import pytest

from parity_util import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2409_05114_gb300 import binding
    return binding


def _lattice(B):
    h, w = B.lbm_velocities()
    h = np.asarray(h, dtype=np.float64).reshape(81, 3)
    return h, np.asarray(w, dtype=np.float64)


def _moments_fp64(f, h):
    """f: [2, 81, sites] dense FP64 -> rho, u [3, ...], theta per site (flattened sub-major)."""
    c = h / 2.0
    rho = f.sum(axis=1)
    j = np.einsum("ia,sin->san", c, f)
    e = np.einsum("i,sin->sn", (c ** 2).sum(axis=1), f)
    u = j / rho[:, None, :]
    theta = (e / rho - (u ** 2).sum(axis=1)) / 3.0
    return rho.reshape(-1), np.moveaxis(u, 1, 0).reshape(3, -1), theta.reshape(-1)


def _run(B, storage, f_dense, nx, ny, nz):
    cfg = B.make_config(nx, ny, nz, 0.1, storage)
    S = 2 * nx * ny * nz
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_set_populations(ctx, f_dense.reshape(-1))
        back = np.zeros(S * 81)
        B.lbm_get_populations(ctx, back)
        r, u, t = np.zeros(S), np.zeros(3 * S), np.zeros(S)
        B.lbm_moments(ctx, r, u, t)
    finally:
        B.lbm_destroy(ctx)
    return back.reshape(f_dense.shape), r, u.reshape(3, S), t


def test_fp32_moments_are_double_word_accurate(B):
    h, w = _lattice(B)
    nx, ny, nz = 64, 16, 8
    n = nx * ny * nz
    rng = np.random.default_rng(81)
    c2 = (h ** 2).sum(axis=1)
    f = np.empty((2, 81, n))
    for key in np.unique(c2):
        dirs = np.flatnonzero(c2 == key)
        ws = w[dirs[0]]
        scale = 2.0 ** (np.floor(np.log2(ws)) - 16)           # w_s ~ 2^16..2^17 units
        m = np.round(ws / scale * (1 + 0.3 * rng.uniform(-1, 1, (2, dirs.size, n))))
        assert np.all(m < 2 ** 18) and np.all(m > 0)
        f[:, dirs] = m * scale
    stored, r, u, t = _run(B, "f32", f, nx, ny, nz)
    np.testing.assert_array_equal(stored, f)                   # exact in FP32
    r0, u0, t0 = _moments_fp64(stored, h)
    assert np.max(np.abs(r / r0 - 1)) < 1e-13
    assert np.max(np.abs(u - u0)) < 1e-13 * np.max(np.abs(u0))
    assert np.max(np.abs(t / t0 - 1)) < 1e-12


def test_fp16_offset_moments(B):
    """Offset path: per site the weighted offset sums round at most 12 times in FP32 (weights
    included), each by 2^-24 of a partial sum bounded by B = sum_i w_i |k_i| |d_i| (k = 1, c_a,
    c^2): the error stays below 1e-6 B, while an FP32 sum of the populations themselves would
    be off by ~1e-7 of rho ~ 1, far above B * 1e-6 ~ 1e-8."""
    h, w = _lattice(B)
    nx, ny, nz = 32, 16, 8
    n = nx * ny * nz
    rng = np.random.default_rng(16)
    d = np.round(rng.uniform(-1, 1, (2, 81, n)) * 2 ** 9) * 2 ** -14   # |d| <= 2^-5, exact in FP16
    f = w.reshape(1, 81, 1) * (1 + d)
    stored, r, u, t = _run(B, "f16", f, nx, ny, nz)
    np.testing.assert_allclose(stored, f, rtol=1e-15, atol=0)
    r0, u0, t0 = _moments_fp64(stored, h)
    c = h / 2.0
    wd = w.reshape(1, 81, 1) * np.abs(d)
    b_r = wd.sum(axis=1).reshape(-1)
    b_j = np.einsum("ia,sin->asn", np.abs(c), wd).reshape(3, -1)
    b_e = np.einsum("i,sin->sn", (c ** 2).sum(axis=1), wd).reshape(-1)
    assert np.all(np.abs(r - r0) <= 1e-6 * b_r)
    assert np.all(np.abs(u - u0) <= 1e-6 * (b_j + np.abs(u0) * b_r) + 1e-15)
    assert np.all(np.abs(t - t0) <= 1e-6 * (b_e + 5 * b_r + b_j.sum(axis=0)))
    assert np.max(b_r) < 0.04                                   # the bound is small: FP32 on rho is not
