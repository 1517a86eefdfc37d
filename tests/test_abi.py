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


STRUCTS = ("swkb_profile", "swkb_domain", "swkb_options", "swkb_plan_info", "swkb_plan_stats",
           "swkb_request", "swkb_server_stats", "swkb_hill_desc", "swkb_batch_options",
           "swkb_batch_info")


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes mirror has the C compiler's size and field offsets: a C
    program built against include/swkb.h prints them (a field name missing
    from the header fails to compile)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "swkb.h"', "int main(void) {"]
    for name in STRUCTS:
        st = getattr(swkb, name)
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in st._fields_:
            lines.append(f'  printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for name in STRUCTS:
        st = getattr(swkb, name)
        assert int(got[name]) == ctypes.sizeof(st), name
        for f in st._fields_:
            assert int(got[f"{name}.{f[0]}"]) == getattr(st, f[0]).offset, (name, f[0])
