"""The ctypes structures of the binding have the layout the C compiler gives the structs of
include/lbm.h (size and every field offset), so arguments cross the boundary intact."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1402_2920_gb300 import lbm as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [B.lbm_eos, B.lbm_params, B.lbm_stats, B.lbm_request, B.lbm_request_result, B.lbm_serve_config]


def _c_layout(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', "int main(void) {"]
    for st in STRUCTS:
        name = st.__name__
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in st._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {" ".join(l.split()[:-1]): int(l.split()[-1]) for l in out.splitlines()}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_ctypes_structs_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for st in STRUCTS:
        name = st.__name__
        assert ctypes.sizeof(st) == c[name + " size"], name
        for f, _ in st._fields_:
            assert getattr(st, f).offset == c["%s %s" % (name, f)], (name, f)
