"""The C-ABI library loads and exports every entry point include/rgx.h declares.

CPU-only: no call here touches a GPU (only the pure host function
rgx_fwd_state_bytes is called).
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rgx.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rgx_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2509_07782_b300 import build_lib
    return build_lib.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("rgx_build_bvh", "rgx_render_forward", "rgx_render_backward", "rgx_scene_create",
                 "rgx_scene_destroy", "rgx_sync_status"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rgx_[a-z0-9_]+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_names_match_header(libpath):
    from paper_2509_07782_b300 import rgx
    assert set(rgx.EXPORTS) == set(declared_symbols())
    assert rgx.rgx_fwd_state_bytes() == 32


def test_struct_layouts_match_the_c_compiler(libpath, tmp_path):
    from paper_2509_07782_b300 import rgx
    src = tmp_path / "layout.c"
    fields = {"rgx_camera": [f for f, _ in rgx.RgxCamera._fields_],
              "rgx_opts": [f for f, _ in rgx.RgxOpts._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rgx.h"', 'int main(void){']
    for st, fs in fields.items():
        lines.append(f'printf("%zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("%zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    vals = [int(v) for v in subprocess.check_output([str(exe)], text=True).split()]
    expect = []
    for cls in (rgx.RgxCamera, rgx.RgxOpts):
        expect.append(ctypes.sizeof(cls))
        expect += [getattr(cls, f).offset for f, _ in cls._fields_]
    assert vals == expect


def test_status_and_flag_constants_match_the_header():
    """Every RGX_* status code and option flag the binding uses has the value
    the header defines, and make_opts sets exactly the flags of the options."""
    from paper_2509_07782_b300 import rgx, synth
    src = open(HEADER).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(RGX_[A-Z0-9_]+)\s+(\d+)\b", src)}
    used = {k: getattr(rgx, k) for k in dir(rgx) if k.startswith("RGX_") and isinstance(getattr(rgx, k), int)}
    assert used and set(used) <= set(defs)
    for k, v in used.items():
        assert defs[k] == v, k
    names = {"skip": "RGX_SKIP", "adaptive": "RGX_ADAPTIVE", "morton": "RGX_MORTON", "ztiles": "RGX_ZTILES",
             "morton63": "RGX_MORTON63"}
    for field, flag in names.items():
        o = synth.Options(**{field: True})
        assert rgx.make_opts(o).flags == defs[flag], field
    assert rgx.make_opts(synth.Options()).flags == 0
    x = rgx.make_opts(synth.fast_options(hit_cap=384, tile_w=16, tile_h=2, max_segments=7, bg=(0.1, 0.2, 0.3)))
    assert (x.hit_cap, x.tile_w, x.tile_h, x.max_segments) == (384, 16, 2, 7)
    assert list(x.bg) == pytest.approx([0.1, 0.2, 0.3])
