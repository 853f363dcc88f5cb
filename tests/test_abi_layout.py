"""The binding's structures have the C header's layout: a C program compiled against
include/rn.h prints the size of every structure the binding declares and the offset of
each of its fields, and the ctypes declarations must agree byte for byte (a field added
on one side only shifts every later one)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _structs():
    from paper_1607_07696_gb300 import rn

    out = []
    for name in dir(rn):
        obj = getattr(rn, name)
        if isinstance(obj, type) and issubclass(obj, C.Structure) and name.startswith("rn_"):
            out.append(obj)
    return out


def test_struct_layouts_match_the_header(tmp_path):
    structs = _structs()
    assert len(structs) >= 13
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rn.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'    printf("{s.__name__} . %zu\\n", sizeof({s.__name__}));')
        for f in s._fields_:
            lines.append(f'    printf("{s.__name__} {f[0]} %zu\\n", offsetof({s.__name__}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    cc = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                        capture_output=True, text=True)
    if cc.returncode != 0:
        pytest.fail("a field the binding declares is missing from the header:\n" + cc.stderr[-3000:])
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        struct, field, value = line.split()
        got[(struct, field)] = int(value)
    for s in structs:
        assert got[(s.__name__, ".")] == C.sizeof(s), f"sizeof({s.__name__})"
        for f in s._fields_:
            assert got[(s.__name__, f[0])] == getattr(s, f[0]).offset, f"{s.__name__}.{f[0]}"


def test_constants_match_the_header(tmp_path):
    """Every RN_ constant the header defines (status codes, flags, bounds, search sides,
    rectangle roles) has the same value in the binding."""
    import re

    from paper_1607_07696_gb300 import rn

    header = open(os.path.join(ROOT, "include", "rn.h")).read()
    names = sorted(set(re.findall(r"#define (RN_[A-Z_]+) ", header)) | set(re.findall(r"^\s+(RN_[A-Z]+) = ", header, re.M)))
    names = [n for n in names if n != "RN_H"]
    assert len(names) >= 15
    lines = ["#include <stdio.h>", '#include "rn.h"', "int main(void) {"]
    lines += [f'    printf("{n} %llu\\n", (unsigned long long)({n}));' for n in names]
    lines += ["    return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, value = line.split()
        assert hasattr(rn, name), f"{name} is missing from the binding"
        assert getattr(rn, name) == int(value), name
