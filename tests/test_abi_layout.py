"""The ctypes mirrors of the C ABI's plain structs (gp_grid, gp_cell,
gp_params, gp_stats) against include/gp.h: the same fields in the same order
with the same types, and the same size and field offsets as the C compiler
lays them out (a small C program built with the host compiler prints them)."""
import os
import re
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

HEADER = os.path.join(ROOT, "include", "gp.h")
STRUCTS = ["gp_grid", "gp_cell", "gp_params", "gp_stats"]


def _binding():
    import ctypes
    from paper_0904_4887_gb300 import gp
    return ctypes, gp


def _header_fields(name):
    """(field, C type, array length or 0) in declaration order."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    consts = {k: int(v) for k, v in re.findall(r"#define\s+(\w+)\s+(\d+)", text)}
    out = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        ctype, names = decl.split(" ", 1)
        for nm in names.split(","):
            nm = nm.strip()
            a = re.fullmatch(r"(\w+)\[(\w+)\]", nm)
            if a:
                n = a.group(2)
                out.append((a.group(1), ctype, consts[n] if n in consts else int(n)))
            else:
                out.append((nm, ctype, 0))
    return out


@pytest.mark.parametrize("name", STRUCTS)
def test_ctypes_fields_match_header(name):
    ctypes, gp = _binding()
    cmap = {"int": ctypes.c_int, "double": ctypes.c_double}
    want = _header_fields(name)
    got = getattr(gp, name)._fields_
    assert [f for f, _ in got] == [f for f, _, _ in want]
    for (f, t), (_, ctype, n) in zip(got, want):
        if n:
            assert t._type_ is cmap[ctype] and t._length_ == n, f
        else:
            assert t is cmap[ctype], f


def test_ctypes_layout_matches_c_compiler():
    ctypes, gp = _binding()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gp.h"', 'int main(void) {']
    for name in STRUCTS:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _, _ in _header_fields(name):
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {}
    for line in out:
        if line:
            s, f, v = line.split()
            c[(s, f)] = int(v)
    for name in STRUCTS:
        cls = getattr(gp, name)
        assert ctypes.sizeof(cls) == c[(name, "size")], name
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == c[(name, f)], (name, f)
