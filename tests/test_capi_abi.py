"""The C ABI library builds, loads and exports every entry point of
include/lbms.h; host-side validation answers without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1809_01600_gb300 import lbms as L

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
HEADER = os.path.join(INCLUDE, "lbms.h")
NET_HEADER = os.path.join(INCLUDE, "lbms_net.h")


def declared_functions(path=HEADER):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbms_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = L.load()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.EXPORTS)


def test_every_network_symbol_is_exported():
    lib = L.load()
    names = declared_functions(NET_HEADER)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.NET_EXPORTS) | set(L.UNET_EXPORTS)


def test_unet_create_rejects_bad_sizes_without_a_gpu():
    """Width and voxel bounds are checked before any CUDA call."""
    lib = L.load()
    h = C.c_void_p()
    for width, vox in ((3, 4096), (33, 4096), (28, 63), (28, L.UNET_MAX_VOXELS + 1)):
        assert lib.lbms_unet_create(width, vox, 0, C.byref(h)) == L.LBMS_EINVAL
        assert not h.value
    assert lib.lbms_unet_create(28, 4096, 0, None) == L.LBMS_EINVAL


def test_bf16_conversion_round_trip():
    x = np.array([0.0, 1.0, -2.5, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 3.0e-3], dtype=np.float32)
    y = L.from_bf16_bits(L.to_bf16_bits(x))
    assert y[0] == 0.0 and y[1] == 1.0 and y[2] == -2.5
    assert y[3] == 1.0                      # tie to even
    assert y[4] == 1.0 + 2 ** -7            # rounds up
    assert abs(y[5] / x[5] - 1.0) < 2 ** -8


def test_default_options_and_status_strings():
    lib = L.load()
    o = L.Options()
    lib.lbms_default_options(C.byref(o))
    assert o.precision == L.LBMS_FP32 and o.coupling == L.LBMS_COUPLING_MS
    assert o.tau_min == 1.0 and o.tau_max == 5.0 and o.check_every == 100
    for s in range(8):
        assert lib.lbms_status_string(s)


def _create(geom_kw=None, species_kw=None, T=1073.0, p=101325.0, opt_kw=None, mask=None):
    lib = L.load()
    if mask is None:
        mask = np.zeros((1, 4, 8), np.uint8)
    gk = dict(dim=2, nx=mask.shape[2], ny=mask.shape[1], nz=mask.shape[0], solid=mask.ctypes.data,
              length_x_m=1e-3, periodic_x=0)
    gk.update(geom_kw or {})
    g = L.Geometry(**gk)
    mm = np.array([2.016, 18.015, 39.948])
    fv = np.array([6.12, 13.1, 16.2])
    nu = np.array([-1, 1, 0], np.int32)
    sk = dict(n=3, molar_mass=L._dptr(mm), fuller_volume=L._dptr(fv),
              stoich=nu.ctypes.data_as(C.POINTER(C.c_int)), electrons=2)
    sk.update(species_kw or {})
    sp = L.Species(**sk)
    df = L.Diffusivities(None, 1e-6, 1.0)
    o = L.Options()
    lib.lbms_default_options(C.byref(o))
    for k, v in (opt_kw or {}).items():
        setattr(o, k, v)
    h = C.c_void_p()
    s = lib.lbms_create(C.byref(g), C.byref(sp), C.byref(df), T, p, C.byref(o), C.byref(h))
    return s, h, lib.lbms_last_error(None).decode()


@pytest.mark.parametrize("geom_kw,species_kw,extra,needle", [
    ({"dim": 4}, None, {}, "dim"),
    ({"nz": 2}, None, {}, "nz must be 1"),
    ({"nx": 2}, None, {}, "nx must be >= 3"),
    ({"solid": None}, None, {}, "solid mask"),
    ({"length_x_m": -1.0}, None, {}, "length_x_m"),
    (None, {"n": 4}, {}, "ternary"),
    (None, {"electrons": 0}, {}, "electrons"),
    (None, None, {"T": -5.0}, "T and p"),
    (None, None, {"opt_kw": {"precision": 7}}, "precision"),
    (None, None, {"opt_kw": {"tau_min": 0.4}}, "tau_min"),
    (None, None, {"opt_kw": {"coupling": 3}}, "coupling"),
    (None, None, {"opt_kw": {"init_mode": 2}}, "init_mode"),
    (None, None, {"opt_kw": {"outlet_bc": 2}}, "outlet_bc"),
    (None, None, {"opt_kw": {"grad_stencil": 2}}, "grad_stencil"),
    (None, None, {"opt_kw": {"outlet_bc": 1, "step_variant": 1}}, "per-cell"),
])
def test_create_rejects_invalid_input(geom_kw, species_kw, extra, needle):
    s, h, msg = _create(geom_kw, species_kw, **extra)
    assert s == L.LBMS_EINVAL
    assert not h.value
    assert needle in msg


def test_create_rejects_blocked_boundary_columns():
    mask = np.zeros((1, 4, 8), np.uint8)
    mask[0, 2, 0] = 1
    s, h, msg = _create(mask=mask)
    assert s == L.LBMS_EINVAL and "columns must be fluid" in msg
    mask = np.ones((1, 4, 8), np.uint8)
    s, h, msg = _create(mask=mask, geom_kw={"periodic_x": 1})
    assert s == L.LBMS_EINVAL and "no fluid" in msg


def test_calls_on_null_handle_fail_cleanly():
    lib = L.load()
    r = C.c_double()
    assert lib.lbms_step(None, 1) == L.LBMS_ESTATE
    assert lib.lbms_residual(None, 1, C.byref(r)) == L.LBMS_ESTATE
    assert lib.lbms_set_bc(None, None, 0.0) == L.LBMS_ESTATE
    lib.lbms_destroy(None)


def test_noalloc_size_bounds_checked_on_the_host():
    """lbms_residual_sums_noalloc refuses n outside [1, INT32_MAX] before any
    CUDA call (the pointers below are never dereferenced): its kernel walks
    the cells with a 64-bit index, so every accepted n is safe."""
    lib = L.load()
    fake = C.c_void_p(0x1000)
    for n in (0, -1, 2 ** 31, 2 ** 40):
        assert lib.lbms_residual_sums_noalloc(fake, fake, n, 0, fake, None) == L.LBMS_EINVAL
    assert lib.lbms_residual_sums_noalloc(None, fake, 5, 0, fake, None) == L.LBMS_EINVAL
    assert lib.lbms_residual_sums_noalloc(fake, None, 5, 0, fake, None) == L.LBMS_EINVAL
    assert lib.lbms_residual_sums_noalloc(fake, fake, 5, 0, None, None) == L.LBMS_EINVAL
