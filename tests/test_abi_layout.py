"""The ctypes mirrors of the C ABI's public structs (paper_2606_03599_gb300/_lib.py) have the
size and field offsets that a C compiler gives the declarations in include/pcband.h.  A field
added to one side only, or in another order, would make the binding read and write the wrong
bytes; this compiles a small C program against the header and compares."""

import ctypes
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "pc_material": "c_material",
    "pc_pcg_info": "c_pcg_info",
    "pc_options": "c_options",
    "pc_eigs_info": "c_eigs_info",
    "pc_batch_job": "c_batch_job",
    "pc_batch_info": "c_batch_info",
    "pc_stats": "c_stats",
}


def _c_layout(tmp_path, mirrors):
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pcband.h"', "int main(void) {",
             '  printf("{");']
    first = True
    for cname, cls in mirrors.items():
        fields = [f[0] for f in cls._fields_]
        sep = "" if first else ","
        first = False
        parts = ['\\"size\\": %zu']
        args = ["sizeof(%s)" % cname]
        for f in fields:
            parts.append('\\"%s\\": %%zu' % f)
            args.append("offsetof(%s, %s)" % (cname, f))
        lines.append('  printf("%s\\"%s\\": {%s}", %s);' % (sep, cname, ", ".join(parts), ", ".join(args)))
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_ctypes_structs_match_the_header(tmp_path):
    from paper_2606_03599_gb300 import _lib
    mirrors = {c: getattr(_lib, py) for c, py in STRUCTS.items()}
    lay = _c_layout(tmp_path, mirrors)
    for cname, cls in mirrors.items():
        got = lay[cname]
        assert got["size"] == ctypes.sizeof(cls), (cname, got["size"], ctypes.sizeof(cls))
        for f in cls._fields_:
            assert got[f[0]] == getattr(cls, f[0]).offset, (cname, f[0], got[f[0]], getattr(cls, f[0]).offset)
