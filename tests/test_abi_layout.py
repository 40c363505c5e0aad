"""The binding's structures have the layout of the C header's (no GPU).

A small C program, compiled with the host compiler against include/lbm.h, prints sizeof and the
offset of every field of each public structure; the ctypes structures of the binding must agree
field by field, so that a change on one side of the boundary without the other fails here
instead of passing garbage through the ABI.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1402_2920_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "lbm_eos": P.lbm_eos,
    "lbm_params": P.lbm_params,
    "lbm_stats": P.lbm_stats,
    "lbm_request": P.lbm_request,
    "lbm_request_result": P.lbm_request_result,
    "lbm_serve_config": P.lbm_serve_config,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


def test_binding_structures_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for name, cls in STRUCTS.items():
        assert layout[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert layout[(name, field)] == getattr(cls, field).offset, (name, field)
