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
