"""The C-ABI library builds, loads and exports every symbol include/csvc.h
declares; host-only entry points answer without a GPU (no device compute)."""
import math
import os

import pytest

from oracle import cs_oracle as O
from paper_1311_1419_gb300 import binding as B
from paper_1311_1419_gb300 import build as build_mod

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_cr.txt")


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    names = B.header_symbols()
    assert "cs_make_phi" in names and "cs_decode_gop" in names and "cs_submit" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []
    # and the binding wraps each of them under the same name
    assert [n for n in names if not callable(getattr(B, n, None))] == []


def test_total_cr_reproduces_table_i(lib):
    for ln in open(GOLDEN):
        if not ln.strip() or ln.startswith("#"):
            continue
        gop, cr_key, cr_cs, want = ln.split()
        assert round(B.cs_total_cr(int(gop), float(cr_key), float(cr_cs)), 2) == float(want)
    assert math.isnan(B.cs_total_cr(0, 23, 40))
    assert math.isnan(B.cs_total_cr(3, -1, 40))


@pytest.mark.parametrize("g,h,w,b,m", [(4, 144, 176, 16, 64), (8, 288, 352, 16, 26),
                                       (16, 720, 1280, 32, 102), (3, 37, 45, 8, 5)])
def test_raw_key_cr_matches_oracle(lib, g, h, w, b, m):
    assert B.cs_raw_key_cr(g, h, w, b, m) == pytest.approx(O.raw_key_cr(g, h, w, b, m), rel=1e-15)


def test_status_strings(lib):
    for st in [B.CS_OK, B.CS_EINVAL, B.CS_ENOMEM, B.CS_EAGAIN, B.CS_ETIMEDOUT, B.CS_ECUDA,
               B.CS_ENOTFOUND, B.CS_ENODEV]:
        assert B.cs_strerror(st)
    assert B.cs_strerror(12345) == "unknown status"


def test_params_struct_matches_header_layout(lib):
    # 10 int32 fields + 1 float, no padding
    assert B.cs_params.__sizeof__(B.make_params(1, 1, 2, 1, 1)) >= 44
    import ctypes
    assert ctypes.sizeof(B.cs_params) == 44
