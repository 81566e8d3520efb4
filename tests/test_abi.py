"""Host-side checks of the C ABI: the library loads and exports every declared entry point."""
import ctypes
import os
import re

import pytest

import paper_2512_13550_gb300 as nof

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "nof.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nof_[a-z_A-Z0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(nof.LIB_PATH):
        from paper_2512_13550_gb300 import build
        build.build()
    return nof.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(nof.SIGNATURES), "binding signatures out of sync with nof.h"


def test_default_options_host_only(lib):
    o = nof.Options()
    lib.nof_default_options(ctypes.byref(o))
    assert (o.ipnof, o.ncwo, o.precision, o.on_iters) == (7, 1, 0, 20)
    assert abs(o.lr - 0.02) < 1e-15 and abs(o.b1 - 0.9) < 1e-15


def test_null_arguments_rejected_without_device_work(lib):
    assert lib.nof_create(None, None, None) == nof.NOF_EINVAL
    assert lib.nof_query(None, None, None, None, None, None) == nof.NOF_EINVAL
    assert lib.nof_destroy(None) == nof.NOF_OK
    assert b"null" in lib.nof_last_error()


def test_argument_checks_of_measurement_and_deployment_entry_points(lib):
    """Invalid arguments are refused on the host, before any device work (no GPU needed)."""
    d = ctypes.c_double(0.0)
    ll = ctypes.c_longlong(0)
    # tile width 24 is not a supported N tile; 5 digits with BN 64 and 4 digits are fine shapes
    assert lib.nof_bench_digit_gemm(128, 64, 24, 4, 10, 10, 0, 1, ctypes.byref(d)) == nof.NOF_EINVAL
    assert lib.nof_bench_digit_gemm(128, 64, 64, 6, 10, 10, 0, 1, ctypes.byref(d)) == nof.NOF_EINVAL
    assert lib.nof_bench_digit_gemm(128, 64, 64, 4, 10, 3, 2, 1, ctypes.byref(d)) == nof.NOF_EINVAL  # chunk % 8
    assert lib.nof_bench_digit_gemm(128, 64, 64, 4, 10, 10, 0, 1, None) == nof.NOF_EINVAL
    assert lib.nof_selftest_digit_gemm(128, 64, 24, 4, 10, 10, 1, ctypes.byref(ll)) == nof.NOF_EINVAL
    assert lib.nof_selftest_digit_gemm(0, 64, 64, 4, 10, 10, 1, ctypes.byref(ll)) == nof.NOF_EINVAL
    assert lib.nof_tuned_tiles(None, (ctypes.c_int * 4)()) == nof.NOF_EINVAL
    assert lib.nof_split_digits(None, ctypes.byref(ctypes.c_int())) == nof.NOF_EINVAL
    # the allocation-free JK refuses sizes beyond its fixed scratch before touching the device
    p = ctypes.c_void_p(16)
    assert lib.nof_jk_static(2000, 600, 200, p, p, p, p, None) == nof.NOF_EINVAL
    assert b"exceeds" in lib.nof_last_error()
    assert lib.nof_jk_static(10, 4, 5, p, p, p, p, None) == nof.NOF_EINVAL  # nact > nbf
    # within the scratch but beyond the transforms' grid limits: refused before anything is queued
    assert lib.nof_jk_static(70000, 1, 1, p, p, p, p, None) == nof.NOF_EINVAL
    assert b"grid limits" in lib.nof_last_error()
    assert lib.nof_jk_static(60000, 80, 1, p, p, p, p, None) == nof.NOF_EINVAL
    # the wait-limit test hook refuses a missing output, a bad tile or a limit outside (0, 1000] ms
    assert lib.nof_selftest_digit_gemm_timeout(128, 64, 64, 4, 4, 2.0, None) == nof.NOF_EINVAL
    assert lib.nof_selftest_digit_gemm_timeout(128, 64, 24, 4, 4, 2.0, ctypes.byref(d)) == nof.NOF_EINVAL
    assert lib.nof_selftest_digit_gemm_timeout(128, 64, 64, 4, 4, 0.0, ctypes.byref(d)) == nof.NOF_EINVAL
    assert lib.nof_selftest_digit_gemm_timeout(128, 64, 64, 4, 4, 5000.0, ctypes.byref(d)) == nof.NOF_EINVAL
    # the converged loop refuses bad parameters before any device work
    prm = nof.OptParams()
    lib.nof_default_opt_params(ctypes.byref(prm))
    assert (prm.maxit, prm.maxloop, prm.gtol, prm.lr, prm.lr_grow) == (1000, 10, 1e-5, 0.02, 1.0)
    res = (ctypes.c_double * 8)()
    assert lib.nof_optimize(None, p, p, ctypes.byref(prm), None, res) == nof.NOF_EINVAL


def test_bad_options_rejected(lib):
    o = nof.Options()
    lib.nof_default_options(ctypes.byref(o))
    assert o.digits == 0
    o.precision, o.digits = 1, 3
    h = ctypes.c_void_p()
    assert lib.nof_create(ctypes.byref(h), ctypes.byref(o), None) == nof.NOF_EINVAL
    o.digits, o.ipnof = 0, 6
    assert lib.nof_create(ctypes.byref(h), ctypes.byref(o), None) == nof.NOF_EINVAL
    lib.nof_default_options(ctypes.byref(o))
    assert o.graphs == 1
    o.graphs = 2
    assert lib.nof_create(ctypes.byref(h), ctypes.byref(o), None) == nof.NOF_EINVAL
    o.graphs, o.isoftmax = 1, 2  # 0 = trigonometric, 1 = softmax mapping
    assert lib.nof_create(ctypes.byref(h), ctypes.byref(o), None) == nof.NOF_EINVAL


def test_misspelt_context_option_is_an_error(lib):
    """Context(**options) names the struct's fields; an unknown name raises before any device
    work instead of being ignored."""
    with pytest.raises(ValueError, match="unknown option 'grpahs'"):
        nof.Context(precision=nof.PREC_SPLIT_BF16, grpahs=0)
