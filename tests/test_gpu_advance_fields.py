"""lbm_advance_fields (init, n steps and moments in one call; pinned host fields staged slab by
slab in z through the copy engines) against lbm_init + lbm_step + lbm_moments.  Both run the same
kernels on the same sites, so the fields agree bitwise: for one slab, several slabs with a ragged
last one, slabs one plane thick (thinner than the pull reach, so most steps wait for slabs across
the periodic z wrap), every x-face kind, n = 0, 1, 2 and 11 (graph replay in between), pinned,
pageable and device fields, outputs that alias the inputs, and the state the context keeps."""

import numpy as np
import pytest

from parity_util import ensure_built
from paper_2409_05114_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

INFLOW = ("eq_inflow", 1.05, 0.2 * W.CS, 0.0, 0.0, 1.02 * W.THETA0)


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2409_05114_gb300 import binding
    return binding


def _fields(wl):
    return (np.ascontiguousarray(wl.rho, dtype=np.float64).reshape(-1),
            np.ascontiguousarray(wl.u, dtype=np.float64).reshape(-1),
            np.ascontiguousarray(wl.theta, dtype=np.float64).reshape(-1))


def _pinned(arrays):
    """Page-locked copies (torch pinned tensors, kept alive) and their numpy views."""
    ts = [torch.from_numpy(a.copy()).pin_memory() for a in arrays]
    return ts, [t.numpy() for t in ts]


def _empty(S, pinned):
    arrs = [np.zeros(S), np.zeros(3 * S), np.zeros(S)]
    return _pinned(arrs) if pinned else (None, arrs)


def _composed(B, cfg, fields, n, more=0):
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_init(ctx, *fields)
        B.lbm_step(ctx, n)
        S = fields[0].size
        out = [np.zeros(S), np.zeros(3 * S), np.zeros(S)]
        B.lbm_moments(ctx, *out)
        after = None
        if more:
            B.lbm_step(ctx, more)
            after = [np.zeros(S), np.zeros(3 * S), np.zeros(S)]
            B.lbm_moments(ctx, *after)
        return out, after
    finally:
        B.lbm_destroy(ctx)


def _fused(B, cfg, fields, n, pinned=True, more=0, alias=False):
    S = fields[0].size
    keep_in, fin = _pinned(fields) if pinned else (None, [a.copy() for a in fields])
    keep_out, fout = (keep_in, fin) if alias else _empty(S, pinned)
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_advance_fields(ctx, *fin, n, *fout)
        out = [a.copy() for a in fout]
        after = None
        if more:
            B.lbm_step(ctx, more)
            after = [np.zeros(S), np.zeros(3 * S), np.zeros(S)]
            B.lbm_moments(ctx, *after)
        return out, after
    finally:
        B.lbm_destroy(ctx)
        del keep_in, keep_out


def _equal(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


GRIDS = {
    # nx, ny, nz, faces: one slab; three slabs of 8, 8 and 4 planes; twelve slabs of one plane
    "one_slab": (16, 12, 10, None),
    "ragged_zg": (256, 256, 20, ["zero_gradient", "zero_gradient"]),
    "ragged_inflow": (256, 256, 20, [INFLOW, "zero_gradient"]),
    "thin": (2048, 256, 12, None),
}


@pytest.mark.parametrize("grid,storage,steps", [
    ("one_slab", "f32", (0, 1, 2, 11)),
    ("one_slab", "f64", (1, 3)),
    ("ragged_zg", "f32", (0, 1, 2)),
    ("ragged_inflow", "f32", (1, 2)),
    ("ragged_zg", "f16", (1,)),
    ("thin", "f32", (1, 2)),
])
def test_fused_equals_separate_calls(B, grid, storage, steps):
    nx, ny, nz, faces = GRIDS[grid]
    wl = W.smooth_random(nx, ny, nz, seed=nz, faces=faces)
    fields = _fields(wl)
    cfg = B.make_config(nx, ny, nz, wl.paper_tau(), storage, wl.faces)
    for n in steps:
        ref, ref_after = _composed(B, cfg, fields, n, more=2)
        got, got_after = _fused(B, cfg, fields, n, more=2)
        _equal(got, ref)
        _equal(got_after, ref_after)       # the context holds the stepped state afterwards


def test_outputs_may_alias_inputs(B):
    nx, ny, nz, faces = GRIDS["ragged_zg"]
    wl = W.smooth_random(nx, ny, nz, seed=3, faces=faces)
    fields = _fields(wl)
    cfg = B.make_config(nx, ny, nz, wl.paper_tau(), "f32", wl.faces)
    for n in (0, 1, 2):
        ref, _ = _fused(B, cfg, fields, n)
        got, _ = _fused(B, cfg, fields, n, alias=True)
        _equal(got, ref)


def test_pageable_and_device_fields(B):
    nx, ny, nz, faces = 64, 48, 20, ["zero_gradient", "zero_gradient"]
    wl = W.smooth_random(nx, ny, nz, seed=5, faces=faces)
    fields = _fields(wl)
    cfg = B.make_config(nx, ny, nz, wl.paper_tau(), "f32", wl.faces)
    ref, _ = _composed(B, cfg, fields, 1)
    got, _ = _fused(B, cfg, fields, 1, pinned=False)
    _equal(got, ref)
    din = [torch.from_numpy(a).cuda() for a in fields]
    dout = [torch.zeros_like(t) for t in din]
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_advance_fields(ctx, *din, 1, *dout)
        torch.cuda.synchronize()
    finally:
        B.lbm_destroy(ctx)
    _equal([t.cpu().numpy() for t in dout], ref)


def test_staged_moments_match_device_moments(B):
    """lbm_moments into pinned host fields (the output ring) against device fields and pageable."""
    nx, ny, nz, faces = GRIDS["ragged_zg"]
    wl = W.smooth_random(nx, ny, nz, seed=9, faces=faces)
    cfg = B.make_config(nx, ny, nz, wl.paper_tau(), "f32", wl.faces)
    S = wl.sites
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_init(ctx, *_fields(wl))
        B.lbm_step(ctx, 3)
        keep, pin = _empty(S, True)
        B.lbm_moments(ctx, *pin)
        page = [np.zeros(S), np.zeros(3 * S), np.zeros(S)]
        B.lbm_moments(ctx, *page)
        dev = [torch.zeros(S, dtype=torch.float64, device="cuda"), torch.zeros(3 * S, dtype=torch.float64, device="cuda"),
               torch.zeros(S, dtype=torch.float64, device="cuda")]
        B.lbm_moments(ctx, *dev)
        torch.cuda.synchronize()
    finally:
        B.lbm_destroy(ctx)
    _equal(pin, page)
    _equal(pin, [t.cpu().numpy() for t in dev])


@pytest.mark.parametrize("grid", ["one_slab", "ragged_inflow", "thin"])
def test_aa_streaming(B, grid):
    """AA contexts pipeline too: neighbour steps per slab in the own layout, moments of the pushed
    layout, the faces' returns after all slabs; n = 3 ends with an own-site step."""
    nx, ny, nz, faces = GRIDS[grid]
    faces = faces and ["zero_gradient", INFLOW]
    wl = W.smooth_random(nx, ny, nz, seed=2, faces=faces)
    fields = _fields(wl)
    cfg = B.make_config(nx, ny, nz, wl.paper_tau(), "f32", wl.faces, streaming="aa")
    for n in ((0, 1, 2, 3) if grid != "thin" else (1, 2)):
        ref, ref_after = _composed(B, cfg, fields, n, more=1)
        got, got_after = _fused(B, cfg, fields, n, more=1)
        _equal(got, ref)
        _equal(got_after, ref_after)


@pytest.mark.parametrize("streaming", ["pingpong", "aa"])
@pytest.mark.parametrize("dims,faces", [((1, 1, 1), None), ((5, 1, 3), None), ((1, 3, 2), None),
                                        ((3, 2, 1), ["zero_gradient", "bounce_back"]),
                                        ((1, 2, 5), ["bounce_back", INFLOW])])
def test_tiny_and_degenerate_grids(B, dims, faces, streaming):
    """One-site rows, planes and grids (every pull wraps onto the same few sites; slabs of one plane
    whose pull reach spans the whole grid) and one-site-wide open channels."""
    wl = W.smooth_random(*dims, seed=sum(dims), mach=0.2, eta=0.03, faces=faces)
    fields = _fields(wl)
    cfg = B.make_config(*dims, wl.paper_tau(), "f32", wl.faces, streaming=streaming)
    for n in (0, 1, 2):
        ref, ref_after = _composed(B, cfg, fields, n, more=1)
        got, got_after = _fused(B, cfg, fields, n, more=1)
        _equal(got, ref)
        _equal(got_after, ref_after)


def test_rejects_bad_arguments(B):
    cfg = B.make_config(8, 8, 8, 0.1, "f32")
    S = 2 * 8 * 8 * 8
    f = [np.ones(S), np.zeros(3 * S), np.full(S, W.THETA0)]
    o = [np.zeros(S), np.zeros(3 * S), np.zeros(S)]
    ctx = B.lbm_create(cfg)
    try:
        with pytest.raises(B.LbmError) as ei:
            B.lbm_advance_fields(ctx, *f, -1, *o)
        assert ei.value.status == B.LBM_EINVAL
        B.lbm_advance_fields(ctx, *f, 1, *o)    # the context is still usable
        np.testing.assert_allclose(o[0], 1.0, rtol=1e-6)
    finally:
        B.lbm_destroy(ctx)
