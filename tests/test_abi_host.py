"""Host-side checks of the C ABI that need no GPU.

* libsphx.so builds for sm_103a, loads, and exports every function that
  include/sphx.h declares;
* every argument error the library promises to catch before a launch comes
  back as SPHX_ERR_INVALID_ARG without touching the device (fake, aligned
  device addresses are never dereferenced);
* without a usable driver, sphx_create fails with a status, not a crash.
"""
import ctypes

import pytest

from paper_2510_09892_gb300 import sphx

FAKE = 1 << 40  # an aligned address that is never dereferenced


def test_library_exports_every_header_symbol():
    L = sphx.lib()
    names = sphx.header_symbols()
    assert "sphx_intersect_gca_constlat" in names and "sphx_intersect_ragged" in names
    for name in names:
        assert hasattr(L, name), name
        assert name in sphx._SIGS, f"binding lacks {name}"


def test_status_strings():
    for st in range(7):
        assert sphx.status_string(st) not in ("", "unknown status")
    assert sphx.status_string(99) == "unknown status"


def test_dense_argument_errors_before_launch():
    L = sphx.lib()
    f = L.sphx_intersect_gca_constlat
    assert f(FAKE, FAKE, FAKE, -1, FAKE, FAKE, 1, None) == sphx.ERR_INVALID_ARG
    assert f(None, FAKE, FAKE, 10, FAKE, FAKE, 1, None) == sphx.ERR_INVALID_ARG
    assert f(FAKE, FAKE, FAKE, 10, FAKE, None, 1, None) == sphx.ERR_INVALID_ARG
    assert f(FAKE + 8, FAKE, FAKE, 10, FAKE, FAKE, 1, None) == sphx.ERR_INVALID_ARG
    assert f(FAKE, FAKE, FAKE, 10, FAKE, FAKE + 4, 1, None) == sphx.ERR_INVALID_ARG
    assert f(FAKE, FAKE, FAKE, 10, FAKE, FAKE, 7, None) == sphx.ERR_INVALID_ARG
    assert f(None, None, None, 0, None, None, 1, None) == sphx.OK  # n = 0: no-op
    h = L.sphx_intersect_gca_constlat_adaptive
    assert h(FAKE, FAKE, FAKE, -1, FAKE, FAKE, 4.0, None, None) == sphx.ERR_INVALID_ARG
    assert h(FAKE, None, FAKE, 10, FAKE, FAKE, 4.0, None, None) == sphx.ERR_INVALID_ARG
    assert h(FAKE, FAKE, FAKE, 10, FAKE + 8, FAKE, 4.0, None, None) == sphx.ERR_INVALID_ARG
    assert h(FAKE, FAKE, FAKE, 10, FAKE, FAKE, 4.0, FAKE + 4, None) == sphx.ERR_INVALID_ARG
    for gate in (0.5, float("nan"), 2.0 ** 27):
        assert h(FAKE, FAKE, FAKE, 10, FAKE, FAKE, gate, None, None) == sphx.ERR_INVALID_ARG
    assert h(None, None, None, 0, None, None, 4.0, None, None) == sphx.OK


def test_adaptive_mode_is_dense_only():
    """The ragged and arc x arc calls refuse the adaptive mode before launching."""
    L = sphx.lib()
    ctx = ctypes.c_void_p(FAKE)
    st = L.sphx_intersect_ragged(ctx, FAKE, FAKE, FAKE, 1, 10, FAKE, FAKE, 5, None, None,
                                 sphx.MODE_ADAPTIVE, FAKE, 10, FAKE, None)
    assert st == sphx.ERR_UNSUPPORTED
    st = L.sphx_intersect_gca_gca(FAKE, FAKE, FAKE, FAKE, 10, FAKE, FAKE, sphx.MODE_ADAPTIVE, None)
    assert st == sphx.ERR_UNSUPPORTED


def test_ragged_argument_errors_before_launch():
    L = sphx.lib()
    f = L.sphx_intersect_ragged
    ctx = ctypes.c_void_p(FAKE)
    # no context
    assert f(None, FAKE, FAKE, FAKE, 1, 10, FAKE, FAKE, 5, None, None, 1, FAKE, 10, FAKE,
             None) == sphx.ERR_INVALID_ARG
    # M < 1, E < 0, bad mode, lo without hi, missing out, unaligned out
    bad = [
        dict(M=0), dict(E=-1), dict(mode=11), dict(lo=FAKE), dict(out=None),
        dict(out=FAKE + 8), dict(total=None), dict(total=FAKE + 4), dict(cap=-1), dict(A=None),
    ]
    base = dict(A=FAKE, B=FAKE, eo=FAKE, M=1, E=10, lz=FAKE, lo_=FAKE, L=5, lo=None, hi=None,
                mode=1, out=FAKE, cap=10, total=FAKE)
    for b in bad:
        a = dict(base, **b)
        st = f(ctx, a["A"], a["B"], a["eo"], a["M"], a["E"], a["lz"], a["lo_"], a["L"], a["lo"],
               a["hi"], a["mode"], a["out"], a["cap"], a["total"], None)
        assert st == sphx.ERR_INVALID_ARG, b
    g = L.sphx_candidate_ranges
    assert g(FAKE, FAKE, FAKE, 0, 10, FAKE, FAKE, 5, FAKE, FAKE, None) == sphx.ERR_INVALID_ARG
    assert g(FAKE, FAKE, FAKE, 1, 10, FAKE, FAKE, 5, None, FAKE, None) == sphx.ERR_INVALID_ARG


def test_band_area_argument_errors_before_launch():
    L = sphx.lib()
    ctx = ctypes.c_void_p(FAKE)
    r = L.sphx_band_ranges
    # no context, too few latitudes, negative sizes, missing outputs
    assert r(None, FAKE, 10, FAKE, FAKE, 40, 10, FAKE, 5, FAKE, FAKE, FAKE, None) == sphx.ERR_INVALID_ARG
    assert r(ctx, FAKE, 10, FAKE, FAKE, 40, 10, FAKE, 1, FAKE, FAKE, FAKE, None) == sphx.ERR_INVALID_ARG
    assert r(ctx, FAKE, 10, FAKE, FAKE, 40, -1, FAKE, 5, FAKE, FAKE, FAKE, None) == sphx.ERR_INVALID_ARG
    assert r(ctx, FAKE, 10, FAKE, FAKE, 40, 10, FAKE, 5, None, FAKE, FAKE, None) == sphx.ERR_INVALID_ARG
    assert r(ctx, FAKE, 10, FAKE, FAKE, 40, 10, FAKE, 5, FAKE, FAKE, None, None) == sphx.ERR_INVALID_ARG
    assert r(ctx, FAKE, 10, FAKE, FAKE, 40, 1 << 31, FAKE, 5, FAKE, FAKE, FAKE, None) == sphx.ERR_INVALID_ARG
    a = L.sphx_band_areas
    assert a(ctx, FAKE, 10, FAKE, FAKE, 40, 10, FAKE, 5, FAKE, FAKE, FAKE, 4, FAKE, -1,
             None) == sphx.ERR_INVALID_ARG
    assert a(ctx, FAKE, 10, FAKE, FAKE, 40, 10, FAKE, 5, FAKE, FAKE, None, 4, FAKE, 10,
             None) == sphx.ERR_INVALID_ARG
    assert a(ctx, None, 10, FAKE, FAKE, 40, 10, FAKE, 5, FAKE, FAKE, FAKE, 4, FAKE, 10,
             None) == sphx.ERR_INVALID_ARG
    z = L.sphx_zonal_sums
    assert z(None, FAKE, FAKE, FAKE, 10, FAKE, FAKE, 5, FAKE, FAKE, None) == sphx.ERR_INVALID_ARG
    assert z(ctx, FAKE, FAKE, FAKE, 10, FAKE, FAKE, 1, FAKE, FAKE, None) == sphx.ERR_INVALID_ARG
    assert z(ctx, FAKE, FAKE, FAKE, 10, FAKE, None, 5, FAKE, FAKE, None) == sphx.ERR_INVALID_ARG


def test_tuning_validation_without_device():
    L = sphx.lib()
    assert L.sphx_set_tuning(None, None) == sphx.ERR_INVALID_ARG
    assert L.sphx_get_tuning(None, None) == sphx.ERR_INVALID_ARG
    assert L.sphx_sync_status(None, None) == sphx.ERR_INVALID_ARG
    assert L.sphx_probe_fma_rate(1, None) == sphx.ERR_INVALID_ARG
    v = ctypes.c_double()
    assert L.sphx_probe_fma_rate(3, ctypes.byref(v)) == sphx.ERR_INVALID_ARG


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = sphx.lib().sphx_create(ctypes.byref(h), 0)
    assert st in (sphx.ERR_CUDA, sphx.ERR_INVALID_ARG, sphx.ERR_UNSUPPORTED)
    assert not h.value
