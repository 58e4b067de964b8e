"""The binding's ctypes structures have the C ABI's layout (CPU only): a
small C program compiled against include/fdsc.h prints each structure's size
and the offset of every field the binding declares, and they must equal
what ctypes computes.  A field the header does not have fails to compile."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2003_05328_gb300 import fdsc as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [("fdsc_params_info", F.ParamsInfo), ("fdsc_layer", F.Layer), ("fdsc_layout", F.Layout),
         ("fdsc_plan_layer", F.PlanLayerC), ("fdsc_plan_layer_info", F.PlanLayerInfo),
         ("fdsc_server_config", F.ServerConfig), ("fdsc_request", F.Request),
         ("fdsc_server_stats", F.ServerStats)]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layouts_match_the_header(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fdsc.h"', "int main(void) {"]
    for cname, py in PAIRS:
        lines.append('printf("%s . %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["return 0;", "}"]
    src, exe = tmp_path / "abi.c", tmp_path / "abi"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines() if ln.strip())}
    for cname, py in PAIRS:
        assert got[(cname, ".")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
