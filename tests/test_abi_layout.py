"""The binding agrees with the C ABI (CPU only).  Structures: a small C
program compiled against include/fdsc.h prints each structure's size and the
offset of every field the binding declares, and they must equal what ctypes
computes (a field the header does not have fails to compile).  Functions:
every prototype in the header has the binding's parameter count, and each
parameter the same kind and width; NULL handles are refused before any
device work."""
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


def _prototypes():
    """name -> (return type, [parameter declarations]) for every function the header declares."""
    import re

    with open(os.path.join(ROOT, "include", "fdsc.h")) as f:
        text = re.sub(r"/\*.*?\*/", " ", f.read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(int|const\s+char\s*\*)\s*(fdsc_\w+)\s*\(([^)]*)\)\s*;", text):
        ret, name, params = m.groups()
        ps = [] if params.strip() in ("", "void") else [" ".join(p.split()) for p in params.split(",")]
        out[name] = (ret, ps)
    return out


def _c_kind(decl: str) -> str:
    if "*" in decl:
        return "ptr"
    ty = decl.replace("const ", "").split()[0]
    return {"uint32_t": "u32", "uint64_t": "u64", "size_t": "u64", "int": "i32", "double": "f64"}[ty]


def _py_kind(t) -> str:
    if t is C.c_void_p or t is C.c_char_p or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    return {C.sizeof(C.c_uint32): "u32", C.sizeof(C.c_uint64): "u64"}[C.sizeof(t)] if t in (
        C.c_uint32, C.c_uint64) else {C.c_int: "i32", C.c_double: "f64"}[t]


def test_binding_signatures_match_the_header():
    """Every function the binding declares exists in fdsc.h with the same
    number of parameters, and each parameter has the same width and kind
    (pointer, 32- or 64-bit unsigned, int, double)."""
    protos = _prototypes()
    assert set(protos) == set(F._SIGS)
    for name, (res, args) in F._SIGS.items():
        assert name in protos, name
        ret, params = protos[name]
        assert (ret == "int") == (res is C.c_int), name
        assert len(params) == len(args), (name, params, args)
        for i, (decl, t) in enumerate(zip(params, args)):
            assert _c_kind(decl) == _py_kind(t), (name, i, decl, t)


def test_null_handles_are_refused_before_any_device_work():
    """Every call whose first parameter is a params, plan or server handle (or
    the plan's layer list, or the server's config) refuses NULL and zero
    arguments with FDSC_ERR_ARG and a message, touching no device (this test
    runs where there is none); the destroy calls accept NULL, as free() does."""
    lib = F.lib()
    handles = ("fdsc_params", "fdsc_plan", "fdsc_server")
    seen = 0
    for name, (ret, params) in sorted(_prototypes().items()):
        if not params or not any(h in params[0] for h in handles):
            continue
        seen += 1
        _, args = F._SIGS[name]
        rc = getattr(lib, name)(*[None if _py_kind(t) == "ptr" else 0 for t in args])
        if name.endswith("_destroy"):
            assert rc == F.FDSC_OK, name
        else:
            assert rc == -1 and lib.fdsc_last_error(), name
    assert seen >= 35
