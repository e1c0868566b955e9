"""The binding's ctypes mirrors of the C structs have the header's layout: a C
program built against include/mdlg.h prints every field offset and the struct
sizes, compared with ctypes' own (no GPU, no library needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1705_04368_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"mdlg_params": binding._Params, "mdlg_stats_out": binding._Stats,
           "mdlg_lattice": binding._Lattice}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mdlg.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for ln in out.splitlines():
        name, key, val = ln.split()
        layout[(name, key)] = int(val)
    return layout


def test_ctypes_structs_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for name, cls in STRUCTS.items():
        assert layout[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert layout[(name, field)] == getattr(cls, field).offset, (name, field)
