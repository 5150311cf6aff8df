"""The ctypes structures of the binding match the C structures of
include/celes.h field by field: a small C program compiled with the host
compiler prints sizeof and every offsetof (CPU only, no GPU)."""

import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1706_02145_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["celes_options", "celes_incident", "celes_solve_opts", "celes_solve_info"]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "celes.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(binding, name)._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        parts = line.split()
        layout[tuple(parts[:-1])] = int(parts[-1])
    return layout


def test_ctypes_structures_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(binding, name)
        assert ctypes.sizeof(cls) == layout[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == layout[(name, field)], (name, field)


def _prototypes():
    import re
    src = open(os.path.join(ROOT, "include", "celes.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    protos = {}
    for m in re.finditer(r"([A-Za-z_][A-Za-z0-9_ \*]*?)\b(celes_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
        ret, name, params = m.group(1).strip(), m.group(2), " ".join(m.group(3).split())
        n = 0 if params in ("", "void") else params.count(",") + 1
        protos[name] = (ret, n)
    return protos


def test_binding_signatures_match_the_prototypes():
    protos = _prototypes()
    assert len(protos) > 30
    for name, res, args in binding.SIGNATURES:
        assert name in protos, name
        ret, n = protos[name]
        assert len(args) == n, (name, len(args), n)
        if ret == "void":
            assert res is None, name
        elif ret == "int":
            assert res is ctypes.c_int, name
