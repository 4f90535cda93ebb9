"""The ctypes structures of the binding have the layout of the header's
structs: a small C program compiled against include/rorbk.h prints every
field's offset and each struct's size, which must equal ctypes' (no GPU)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2510_02156_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "rorbk_matrix": B.Matrix,
    "rorbk_partition": B.Partition,
    "rorbk_trace": B.Trace,
    "rorbk_options": B.Options,
    "rorbk_result": B.Result,
    "rorbk_info": B.Info,
    "rorbk_tuning": B.Tuning,
}
# ctypes names that differ from the C member (a Python keyword)
RENAMED = {"lambda_": "lambda"}


def _c_layout(tmp_path):
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rorbk.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'printf("{cname} . %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            cf = RENAMED.get(fname, fname)
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines())}


def test_binding_structs_match_the_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lay = _c_layout(tmp_path)
    for cname, cls in STRUCTS.items():
        assert lay[(cname, ".")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert lay[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
