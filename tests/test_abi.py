"""The C-ABI library (CPU-side checks, no device compute): it builds, loads, exports every
entry point include/lbm.h declares, reports the RD3Q81 velocity set the oracle builds
independently, and validates configurations on the host (lbm_footprint)."""

import os
import re

import numpy as np
import pytest

from parity_util import ROOT, ensure_built, lib_perm
from oracle import rd3q81 as O


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2409_05114_gb300 import binding
    return binding


def _declared():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)          # drop comments
    return sorted(set(re.findall(r"^\s*(?:lbm_status|int|const char\s*\*)\s*(lbm_[a-z_0-9]+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(B):
    import ctypes
    lib = ctypes.CDLL(B.library_path())
    names = _declared()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_velocity_set_matches_oracle(B):
    h, w = B.lbm_velocities()
    lat = O.velocity_set()
    perm = lib_perm()
    assert sorted(perm.tolist()) == list(range(81))
    np.testing.assert_array_equal(h, lat.h[perm])
    np.testing.assert_allclose(w, lat.w[perm], rtol=1e-13, atol=0)  # FP64 Horner of the table rows
    # +/- pairs are adjacent: direction 2k is -direction 2k-1
    np.testing.assert_array_equal(h[2::2], -h[1::2])


def _cfg(B, **kw):
    args = dict(nx=16, ny=8, nz=4, tau=0.1, storage="f32")
    args.update(kw)
    faces = args.pop("faces", None)
    return B.make_config(faces=faces, **args)


def test_footprint_and_padding(B):
    n = 64 * 32 * 8
    fp = B.lbm_footprint(_cfg(B, nx=64, ny=32, nz=8))
    assert fp >= 2 * 2 * 81 * n * 4
    assert fp < 2 * 2 * 81 * n * 4 * 1.05 + (64 << 20)
    fp16 = B.lbm_footprint(_cfg(B, nx=64, ny=32, nz=8, storage="f16"))
    fp64 = B.lbm_footprint(_cfg(B, nx=64, ny=32, nz=8, storage="f64"))
    assert fp16 < fp < fp64
    # non-periodic x adds aligned ghost layers
    fz = B.lbm_footprint(_cfg(B, nx=64, ny=32, nz=8, faces=["zero_gradient", "zero_gradient"]))
    assert fz > fp


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(ny=-1), dict(tau=-0.1), dict(tau=float("nan")), dict(storage=7),
    dict(faces=["periodic", "zero_gradient"]),
    dict(faces=["periodic", "periodic", "zero_gradient"]),
    dict(faces=[("eq_inflow", -1.0, 0, 0, 0, 0.8), "zero_gradient"]),
    dict(faces=[("eq_inflow", 1.0, 0, 0, 0, 0.0), "zero_gradient"]),
    dict(nx=2048, ny=2048, nz=1024),
])
def test_invalid_configs_rejected(B, bad):
    with pytest.raises(B.LbmError) as ei:
        B.lbm_footprint(_cfg(B, **bad))
    assert ei.value.status == B.LBM_EINVAL
    assert B.lbm_last_error(None) != "no error"


def test_bad_face_kind_rejected(B):
    cfg = _cfg(B)
    cfg.face[0].kind = 9
    with pytest.raises(B.LbmError):
        B.lbm_footprint(cfg)
    cfg = _cfg(B)
    cfg.velset = 2
    with pytest.raises(B.LbmError):
        B.lbm_footprint(cfg)


def test_equilibrium_and_collision_validation(B):
    for kw in (dict(equilibrium="entropic", collision="entropic"), dict(equilibrium="series_exact_w"),
               dict(equilibrium="series", fp64_moments=True), dict(fp64_moments=True, streaming="aa")):
        assert B.lbm_footprint(B.make_config(16, 8, 4, 0.1, "f32", **kw)) > 0
    for kw in (dict(equilibrium="series", collision="entropic"),            # alpha needs the exact equilibrium
               dict(equilibrium="series_exact_w", collision="entropic"),
               dict(equilibrium="entropic", collision=5),
               dict(equilibrium=3),
               dict(equilibrium="entropic", fp64_moments=True),
               dict(equilibrium="series_exact_w", fp64_moments=True)):
        with pytest.raises(B.LbmError) as ei:
            B.lbm_footprint(B.make_config(16, 8, 4, 0.1, "f32", **kw))
        assert ei.value.status == B.LBM_EINVAL


def test_null_context_calls_are_einval(B):
    import ctypes
    lib = B._lib
    assert lib.lbm_step(None, 1) == B.LBM_EINVAL
    assert lib.lbm_sync(None) == B.LBM_EINVAL
    assert lib.lbm_destroy(None) == B.LBM_EINVAL
    assert lib.lbm_totals(None, None) == B.LBM_EINVAL
    assert lib.lbm_advance_fields(None, None, None, None, 1, None, None, None, 0) == B.LBM_EINVAL
    assert lib.lbm_last_error(None) is not None


def test_bounce_back_faces_validated(B):
    """The bounce-back wall (the Sod setup of Sec. IV A) is an x-face kind: accepted on either x
    face, alone or beside zero-gradient or inflow, with ghost layers like the other open kinds;
    rejected on y and z faces and when paired with a periodic x face."""
    ok = [["bounce_back", "bounce_back"], ["bounce_back", "zero_gradient"],
          [("eq_inflow", 1.0, 0.1, 0, 0, 0.8), "bounce_back"]]
    periodic = B.lbm_footprint(_cfg(B, nx=64))
    for faces in ok:
        fp = B.lbm_footprint(_cfg(B, nx=64, faces=faces))
        assert fp > periodic                                    # ghost layers padded into every row
    for faces in (["bounce_back", "periodic"], ["periodic", "bounce_back"],
                  ["periodic", "periodic", "bounce_back"], ["periodic"] * 5 + ["bounce_back"]):
        with pytest.raises(B.LbmError) as ei:
            B.lbm_footprint(_cfg(B, faces=faces))
        assert ei.value.status == B.LBM_EINVAL


def test_footprint_counts_the_staging_ring(B):
    """lbm_footprint covers the populations plus the host-transfer staging ring: two rings of 3 slots
    of 10 FP64 rows of a z slab (about 2^20 sites per sublattice, whole planes), so at 512^2 x 8
    planes the ring adds ~503 MB beyond one buffer pair, and AA halves only the populations."""
    pp = B.lbm_footprint(_cfg(B, nx=512, ny=512, nz=8))
    aa = B.lbm_footprint(_cfg(B, nx=512, ny=512, nz=8, streaming="aa"))
    pops = 2 * 81 * 512 * 512 * 8 * 4                          # one buffer, both sublattices, FP32
    assert pp - aa >= pops                                      # AA drops one buffer
    ring = 2 * 3 * 10 * (4 * 512 * 512) * 8                     # 4 planes of 512^2 per slab
    assert pp >= 2 * pops + ring
    assert pp < 2 * pops * 1.01 + ring + (200 << 20)


def test_advance_fields_null_arguments_are_einval(B):
    lib = B._lib
    assert lib.lbm_advance_fields(None, None, None, None, 0, None, None, None, 1) == B.LBM_EINVAL
    with pytest.raises(ValueError):
        B.lbm_advance_fields(None, np.zeros(2), np.zeros(6), np.zeros(2), 1,
                             np.zeros(2), np.zeros(6), np.zeros(2, dtype=np.float32))
