"""The binding's ctypes structures match the C ABI's structs in include/xdg.h: same field names,
offsets and sizes (a field added to one side only would shift every later field silently).
A small C program, generated from the ctypes field lists and compiled with the system C
compiler against the header, prints sizeof and offsetof of every struct and field. No GPU.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2003_02431_gb300 import xdg

PAIRS = [
    (xdg.Problem, "xdg_problem"),
    (xdg.HierOpts, "xdg_hier_opts"),
    (xdg.SolveOpts, "xdg_solve_opts"),
    (xdg.SolveInfo, "xdg_solve_info"),
    (xdg.HierInfo, "xdg_hier_info"),
    (xdg.BatchResult, "xdg_batch_result"),
    (xdg.BatchInfo, "xdg_batch_info"),
    (xdg.TrainOpts, "xdg_train_opts"),
    (xdg.SchwarzInfo, "xdg_schwarz_info"),
    (xdg.OrthoMGOpts, "xdg_orthomg_opts"),
    (xdg.GmresOpts, "xdg_gmres_opts"),
]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_ctypes_structs_match_header(tmp_path):
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "xdg.h"', "int main(void) {"]
    for cls, cname in PAIRS:
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", inc, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for cls, cname in PAIRS:
        assert int(got["%s sizeof" % cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got["%s.%s" % (cname, fname)]) == getattr(cls, fname).offset, (cname, fname)
