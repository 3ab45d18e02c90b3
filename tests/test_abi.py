"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b((?:nla|kt)_[A-Za-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libnla():
    from paper_2608_21227_gb300 import _build

    return ctypes.CDLL(_build.build())


def test_headers_declare_entry_points():
    names = declared_symbols()
    for required in ("nla_gesvd_vals", "nla_gesvd_vals_batched", "nla_gebrd_band", "nla_band2bd",
                     "nla_bdsvd_vals", "nla_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libnla):
    missing = [s for s in declared_symbols() if not hasattr(libnla, s)]
    assert not missing, f"not exported: {missing}"


def test_argument_errors_without_gpu(libnla):
    # argument checks return synchronously and touch no device
    libnla.nla_last_error.restype = ctypes.c_char_p
    assert libnla.nla_gesvd_vals(-1, 4, 0, None, 4, None, None, 0, None, None, None) == 1
    assert b"negative" in libnla.nla_last_error()
    assert libnla.nla_gesvd_vals(4, 4, 9, None, 4, None, None, 0, None, None, None) == 1
    b = ctypes.c_size_t(0)
    assert libnla.nla_gebrd_band_workspace(3, 5, 2, 0, None, ctypes.byref(b)) == 1
