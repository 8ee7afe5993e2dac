"""The ctypes mirrors of the C-ABI structs in the Python binding have the
layout include/tl.h gives them: a small C program compiled with the host
compiler prints sizeof of each struct and offsetof of each field the binding
names (a name the header lacks fails to compile), and the binding's ctypes
offsets and sizes must be the same.  No GPU and no CUDA toolkit needed."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ("tl_material", "tl_params", "tl_newton_stats", "tl_mesh_info", "tl_timing", "tl_adamw_params",
           "tl_adamw_stats", "tl_tune_result")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no host C compiler")
def test_ctypes_mirrors_match_the_header_layout():
    from paper_2604_10357_gb300 import tl
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tl.h"', "int main(void) {"]
    expect = {}
    for name in STRUCTS:
        cls = getattr(tl, name)
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        expect[name] = ctypes.sizeof(cls)
        for field, _ in cls._fields_:
            if field.startswith("_pad"):
                continue                   # explicit padding in the mirror: the C struct's implicit padding
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
            expect[f"{name}.{field}"] = getattr(cls, field).offset
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = {k: int(v) for k, v in (line.split() for line in out.strip().splitlines())}
    bad = {k: (got[k], expect[k]) for k in expect if got[k] != expect[k]}
    assert not bad, bad
