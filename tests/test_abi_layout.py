"""The binding's ctypes structures against the C ABI's structs (include/sofa.h).

For every struct that crosses the boundary, the field names are read from the
header in declaration order and must equal the ctypes `_fields_` names.  A
small C program compiled against the header then prints each field's offset
and the struct's size, and those must equal the ctypes layout.  This catches a
field added, removed or reordered on one side only, including a trailing
32-bit field that the struct's padding would hide from a size check alone.
CPU only: gcc and the header, no library call.
"""
import os
import re
import shutil
import subprocess

import pytest

from paper_2411_17483_gb300 import sofa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sofa.h")

PAIRS = [
    ("sofa_build_opts", sofa.BuildOpts),
    ("sofa_train_opts", sofa.TrainOpts),
    ("sofa_tuning", sofa.Tuning),
    ("sofa_stats_t", sofa.Stats),
    ("sofa_profile_t", sofa.Profile),
    ("sofa_info_t", sofa.Info),
]


def header_fields(name):
    """Field names of `typedef struct { ... } name;` in declaration order."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    m = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + re.escape(name) + r"\s*;", text)
    assert m, f"struct {name} not found in the header"
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = [p.strip() for p in decl.split(",")]
        for i, part in enumerate(parts):
            part = re.sub(r"\[[^\]]*\]", "", part).replace("*", " ")
            ident = re.findall(r"[A-Za-z_]\w*", part)
            assert ident, f"cannot read a field of {name} from {decl!r}"
            names.append(ident[-1])
    return names


@pytest.mark.parametrize("cname,cls", PAIRS, ids=[p[0] for p in PAIRS])
def test_field_names_match_the_header(cname, cls):
    assert [f[0] for f in cls._fields_] == header_fields(cname)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_offsets_and_sizes_match_the_header(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sofa.h"', "int main(void) {"]
    for cname, cls in PAIRS:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in header_fields(cname):
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {}
    for line in out:
        if line:
            s, f, v = line.split()
            c[(s, f)] = int(v)
    import ctypes
    for cname, cls in PAIRS:
        assert c[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert c[(cname, f)] == getattr(cls, f).offset, (cname, f)
