"""The C-ABI library builds, loads and exports every function that
include/hdfilter.h declares; argument errors are reported before any device
work.  CPU only: no call here reaches the GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1811_02363_gb300 import build
    build.build()
    from paper_1811_02363_gb300 import _lib
    return _lib


def _declared():
    src = open(os.path.join(ROOT, "include", "hdfilter.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdf_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound(L):
    names = _declared()
    assert "hdf_apply" in names and "hdf_create" in names
    bound = {s[0] for s in L.SIGNATURES}
    for name in names:
        assert hasattr(L.lib(), name), name
        assert name in bound, name


def test_argument_errors_without_device_work(L):
    lib = L.lib()
    d = L.hdf_desc(H=8, W=8, n=3, rho=3, K=4, S=0, sigma_s=1.0, sigma_r=0.1,
                   guide_dtype=0, coef=0)
    h = C.c_void_p()
    bad = L.hdf_desc.from_buffer_copy(d)
    bad.H = 0
    assert lib.hdf_create(C.byref(h), C.byref(bad)) == L.HDF_EINVAL
    bad = L.hdf_desc.from_buffer_copy(d)
    bad.sigma_r = -1.0
    assert lib.hdf_create(C.byref(h), C.byref(bad)) == L.HDF_EINVAL
    bad = L.hdf_desc.from_buffer_copy(d)
    bad.K = L.HDF_MAX_K + 1
    assert lib.hdf_create(C.byref(h), C.byref(bad)) == L.HDF_EUNSUPPORTED
    bad = L.hdf_desc.from_buffer_copy(d)
    bad.S = L.HDF_MAX_S + 1
    assert lib.hdf_create(C.byref(h), C.byref(bad)) == L.HDF_EUNSUPPORTED
    bad = L.hdf_desc.from_buffer_copy(d)
    bad.spatial = 7
    assert lib.hdf_create(C.byref(h), C.byref(bad)) == L.HDF_EINVAL
    assert lib.hdf_bruteforce(C.byref(bad), None, None, None, None) == L.HDF_EINVAL
    assert lib.hdf_bruteforce(C.byref(d), None, None, None, None) == L.HDF_EINVAL
    assert lib.hdf_apply(None, None, None, None, None) == L.HDF_EINVAL
    assert lib.hdf_status_string(L.HDF_ETIMEOUT).startswith(b"HDF_ETIMEOUT")


@pytest.mark.parametrize("field,value,status", [
    ("W", 0, "HDF_EINVAL"), ("n", 0, "HDF_EINVAL"), ("rho", 0, "HDF_EINVAL"),
    ("K", 0, "HDF_EINVAL"), ("sigma_s", 0.0, "HDF_EINVAL"), ("sigma_s", float("nan"), "HDF_EINVAL"),
    ("sigma_r", float("inf"), "HDF_EINVAL"), ("S", -1, "HDF_EINVAL"), ("guide_dtype", 2, "HDF_EINVAL"),
    ("coef", 2, "HDF_EINVAL"), ("rho", 10 ** 6, "HDF_EUNSUPPORTED"), ("n", 10 ** 6, "HDF_EUNSUPPORTED"),
    ("H", 1 << 20, "HDF_EUNSUPPORTED"),   # H * W beyond the pixel limit
])
def test_each_invalid_field_is_reported(L, field, value, status):
    lib = L.lib()
    d = L.hdf_desc(H=8, W=1 << 12, n=3, rho=3, K=4, S=0, sigma_s=1.0, sigma_r=0.1,
                   guide_dtype=0, coef=0)
    setattr(d, field, value)
    h = C.c_void_p()
    assert lib.hdf_create(C.byref(h), C.byref(d)) == getattr(L, status)
    assert lib.hdf_bruteforce(C.byref(d), None, None, None, None) in (L.HDF_EINVAL,
                                                                     getattr(L, status))


def test_recursive_gaussian_needs_sigma_half(L):
    lib = L.lib()
    d = L.hdf_desc(H=8, W=8, n=3, rho=3, K=4, S=0, sigma_s=0.4, sigma_r=0.1,
                   guide_dtype=0, coef=0, spatial=L.HDF_SPATIAL_YOUNG)
    h = C.c_void_p()
    assert lib.hdf_create(C.byref(h), C.byref(d)) == L.HDF_EINVAL


def test_batch_argument_errors_without_device_work(L):
    lib = L.lib()
    d = (L.hdf_desc * 2)()
    for i in range(2):
        d[i] = L.hdf_desc(H=8 + i, W=8, n=3, rho=3, K=4, S=0, sigma_s=1.0, sigma_r=0.1,
                          guide_dtype=0, coef=0)
    b = C.c_void_p()
    assert lib.hdf_batch_create(C.byref(b), 0, d) == L.HDF_EINVAL
    assert lib.hdf_batch_create(C.byref(b), 2, None) == L.HDF_EINVAL
    d[1].sigma_s = 0.0
    assert lib.hdf_batch_create(C.byref(b), 2, d) == L.HDF_EINVAL
    d[1].sigma_s = 1.0
    d[1].S = L.HDF_MAX_S + 1
    assert lib.hdf_batch_create(C.byref(b), 2, d) == L.HDF_EUNSUPPORTED
    assert lib.hdf_batch_run(None, 0, None) == L.HDF_EINVAL
    assert lib.hdf_batch_bind(None, None, None, None) == L.HDF_EINVAL
    assert lib.hdf_batch_tune(None, 3, None) == L.HDF_EINVAL
    assert lib.hdf_batch_get_info(None, None) == L.HDF_EINVAL



@pytest.mark.parametrize("field,value,status", [
    ("sigma_s", float("inf"), "HDF_EINVAL"),
    ("sigma_s", 1e10, "HDF_EUNSUPPORTED"),     # S = ceil(3 sigma_s) would not fit HDF_MAX_S
    ("sigma_s", 11.0, "HDF_EUNSUPPORTED"),     # S = 33
    ("spatial", 7, "HDF_EINVAL"),
])
def test_sigma_and_spatial_checks_before_any_work(L, field, value, status):
    """hdf_create and hdf_apply_static share one descriptor check: an infinite
    or huge sigma_s and an unknown spatial kernel are refused before anything
    is allocated or enqueued."""
    import torch
    lib = L.lib()
    d = L.hdf_desc(H=8, W=8, n=3, rho=3, K=4, S=0, sigma_s=1.0, sigma_r=0.1,
                   guide_dtype=0, coef=0)
    setattr(d, field, value)
    h = C.c_void_p()
    assert lib.hdf_create(C.byref(h), C.byref(d)) == getattr(L, status)
    if torch.cuda.is_available():
        return   # the static call below passes placeholder pointers: host without a GPU only
    dummy = C.c_void_p(256)
    out = C.c_void_p(512)
    assert lib.hdf_apply_static(C.byref(d), dummy, 4, dummy, dummy, out, None) == \
        getattr(L, status)
