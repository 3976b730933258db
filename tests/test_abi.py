"""The C-ABI library builds, loads without a GPU, and exports every call include/mdc.h declares.

No compute call is made here (no device in the CPU test run); host-only helpers
(mdc_kernel_bytes, mdc_strerror) are checked against Table 1 of the paper.
"""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"^\s*typedef[^;]*;", "", text, flags=re.M | re.S)      # function-pointer types
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\*?\s*(\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2011_11120_gb300 import build
    build.build()
    import paper_2011_11120_gb300 as m
    return m


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mdc_create", "mdc_forward", "mdc_adjoint", "marchenko_lsqr", "mdc_destroy",
                     "mdc_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in lib.SIGNATURES, f"binding lacks {name}"


def test_strerror_and_null_handle_without_device(lib):
    L = lib.lib()
    assert L.mdc_strerror(0) == b"ok"
    assert L.mdc_strerror(-1) == b"invalid argument"
    assert L.mdc_forward(None, None, None, 1, 0, None) == -1
    assert L.mdc_destroy(None) == -1
    h = ctypes.c_void_p()
    assert L.mdc_create(ctypes.byref(h), None, 10, 5, 5, 64, 0.004, 1.0, 0, None) == -1
    # argument checks come before any device call
    assert L.mdc_create_empty(ctypes.byref(h), 40, 5, 5, 64, 0.004, 1.0, 0, None) == -1   # nfmax > nt/2 + 1
    assert L.mdc_create_empty(ctypes.byref(h), 10, 5, 5, 100, 0.004, 1.0, 0, None) == -1  # nt not a power of 2
    assert L.mdc_create_empty(ctypes.byref(h), 10, 5, 5, 64, 0.004, 1.0, 9, None) == -1   # unknown storage
    assert L.mdc_load_slab(None, None, 0, 1, None) == -1


def test_kernel_bytes_reproduce_table1(lib):
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "table1_kernel_sizes.json")))
    for row in gold["rows"]:
        n, nf = row["n"], row["nf"]
        # the library pads rows to 64 complex; the paper's figure is the unpadded array
        unpadded = nf * n * n * 8
        assert abs(unpadded / 1e9 - row["kernel_gb"]) <= 0.02 * row["kernel_gb"] + 0.5
        assert abs(row["nt"] * n * n * 4 / 1e9 - row["data_gb"]) <= 0.02 * row["data_gb"] + 0.5
        padded = lib.mdc_kernel_bytes(nf, n, n, "c64")
        assert unpadded <= padded <= unpadded * (1 + 64.0 / n)
        assert lib.mdc_kernel_bytes(nf, n, n, "c16f") < padded // 2 + nf * n * 4 + 1
