"""The ctypes mirrors of the C ABI's structs have the C compiler's layout:
a small C program built with gcc against include/sng.h prints sizeof and
offsetof of every field, and the Python mirrors must agree field by field
(catches a field added on one side only, or reordered)."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2006_06743_gb300 as sng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["sng_params", "sng_stats", "sng_graph", "sng_mi_terms", "sng_mlp_config",
           "sng_gate"]


def _c_layout(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sng.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(sng, name)
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr      # a Python-only field fails to compile here
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


def test_ctypes_mirrors_match_the_c_layout(tmp_path):
    c = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(sng, name)
        assert ctypes.sizeof(cls) == c[(name, "sizeof")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == c[(name, field)], (name, field)
