"""lbm_totals_noalloc: the conservation sums for callers that cannot allocate device memory
(their own memory pool already holds the device's free memory, or they must not let
cudaMalloc/cudaFree synchronise the device).  Called through the C-ABI, it must agree with
lbm_totals on the same populations, call after call, and reject grids larger than its
fixed scratch array.  Kept in the last-collected file so that a stop-at-first-failure run
has run every other test before it."""

import ctypes

import numpy as np
import pytest

from parity_util import ensure_built
from paper_2409_05114_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2409_05114_gb300 import binding
    fn = binding._lib.lbm_totals_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return binding


_TORCH_TYPE = {"f64": "float64", "f32": "float32", "f16": "float16", "bf16": "bfloat16"}


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_noalloc_totals_match_lbm_totals(B, storage):
    import torch
    wl = W.smooth_random(24, 12, 10, seed=21, mach=0.4, eta=0.05)
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, 0.1, storage)
    ctx = B.lbm_create(cfg)
    try:
        B.lbm_init(ctx, wl.rho.reshape(-1).copy(), wl.u.reshape(-1).copy(), wl.theta.reshape(-1).copy())
        B.lbm_step(ctx, 3)
        ref = B.lbm_totals(ctx)
        f = torch.empty(2 * 81 * wl.nx * wl.ny * wl.nz, dtype=torch.float64, device="cuda")
        B.lbm_get_populations(ctx, f)
    finally:
        B.lbm_destroy(ctx)
    # The caller's own buffer in the storage type.  lbm_get_populations decodes the stored
    # values exactly into FP64, so converting back recovers them: FP32 values directly, offset
    # types as d = f/w - 1 (round to nearest recovers the stored d).
    dt = getattr(torch, _TORCH_TYPE[storage])
    if storage in ("f16", "bf16"):
        w = torch.tensor(B.lbm_velocities()[1], dtype=torch.float64, device="cuda")
        fin = (f.view(2, 81, -1) / w.view(1, 81, 1) - 1.0).reshape(-1).to(dt)
    else:
        fin = f.to(dt)
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    code = B.STORAGE[storage]
    # both sides sum the same stored values in FP64 (in different orders)
    tol = 1e-13
    scale = np.array([ref[0]] * 4 + [ref[4]])
    for _ in range(2):
        out.fill_(float("nan"))
        st = B._lib.lbm_totals_noalloc(fin.data_ptr(), code, wl.nx, wl.ny, wl.nz, out.data_ptr(), None)
        assert st == B.LBM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= tol * scale), (got, ref)


def test_noalloc_rejects_grids_beyond_its_scratch(B):
    import torch
    f = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    # 2 * 256^3 = 33,554,432 sites is the largest grid its 4096 partial sums cover
    st = B._lib.lbm_totals_noalloc(f.data_ptr(), B.LBM_F32, 256, 256, 257, out.data_ptr(), None)
    assert st == B.LBM_EINVAL
    assert B._lib.lbm_totals_noalloc(None, B.LBM_F32, 4, 4, 4, out.data_ptr(), None) == B.LBM_EINVAL
    torch.cuda.synchronize()
    assert torch.all(out == 0)
