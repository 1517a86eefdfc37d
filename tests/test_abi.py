"""The C-ABI library builds, loads and exports every symbol of include/swkb.h
(no GPU needed: nothing here launches device work)."""
import ctypes
import os
import re

import pytest

from paper_2301_03814_gb300 import swkb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(swkb.LIB_PATH):
        from paper_2301_03814_gb300 import build
        build.build()
    return ctypes.CDLL(swkb.LIB_PATH)


def header_functions():
    src = open(os.path.join(ROOT, "include", "swkb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(swkb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("swkb_plan_create", "swkb_propagate", "swkb_submit", "swkb_poll",
                 "swkb_server_create", "swkb_plan_destroy", "swkb_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    for name in header_functions():
        assert hasattr(built, name), name
    assert set(swkb.EXPORTED) <= set(header_functions())


def test_status_strings_and_defaults(built):
    swkb._lib = None
    L = swkb.lib()
    assert L.swkb_status_string(0) == b"ok"
    assert L.swkb_status_string(3) == b"caustic between screens"
    o = swkb.swkb_options_default()
    assert o.precision == swkb.SWKB_FP64 and o.ray_stride == 1 and o.rk4_steps == 8


def test_struct_layouts_match_header():
    # sizes of the C structs as laid out by a C compiler for this ABI (LP64)
    assert ctypes.sizeof(swkb.swkb_domain) == 32
    assert ctypes.sizeof(swkb.swkb_profile) == 64
    assert ctypes.sizeof(swkb.swkb_options) == 64
