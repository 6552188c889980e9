"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/biglasso_gpu.h declares.  No compute call is made (no GPU needed):
only entry points that fail argument checks on the host before touching CUDA."""
import ctypes as C
import os
import re
import subprocess

from paper_1701_05936_gb300 import bl, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    L = bl.lib()
    syms = bl.header_symbols()
    assert len(syms) >= 14
    missing = [s for s in syms if not hasattr(L, s)]
    assert missing == []
    assert "sm_103a" in bl.version()


def test_every_entry_point_is_documented_with_a_citation_or_role():
    text = open(os.path.join(ROOT, "include", "biglasso_gpu.h")).read()
    for name in bl.header_symbols():
        m = re.search(r"/\*(?:(?!\*/).)*\*/\s*(?:const\s+)?\w+\s*\*?\s*" + name + r"\s*\(", text, flags=re.S)
        assert m, f"{name} has no comment block directly above its declaration"


def test_host_side_argument_checks_need_no_gpu():
    L = bl.lib()
    # NULL context and NULL arguments are rejected before any CUDA call
    assert L.bl_fit_path(None, None, 1, 10, 10, 16, None, None, None, 10, None) == bl.BL_ERR_ARG
    assert L.bl_standardize(None, None, 1, 10, 10, 16, None, None, None, None) == bl.BL_ERR_ARG
    assert L.bl_cd_active(None, None, 1, 10, 10, 16, None, None, None, 0, 0.1, 1.0, None, None, 1e-7, 10,
                          None) == bl.BL_ERR_ARG
    assert L.bl_ctx_destroy(None) == bl.BL_ERR_ARG
    assert L.bl_ctx_create(None, 0, None) == bl.BL_ERR_ARG
    assert L.bl_last_error(None) == b"null context"
    # the persistent many-problem form: argument checks and its launch-shape table
    assert L.bl_fit_many_persistent(None, None, 1, None, -1) == bl.BL_ERR_ARG
    assert L.bl_many_autotune(None, None, 1, None, None, None) == bl.BL_ERR_ARG
    assert L.bl_many_phase_ms(None, None, 0) == bl.BL_ERR_ARG
    assert L.bl_many_problem_ms(None, None, 0) == bl.BL_ERR_ARG
    shapes = bl.bl_many_configs()
    assert len(shapes) == L.bl_many_num_configs() == 4
    assert all(s and "threads" in s for s in shapes)
    assert L.bl_many_config_name(-1) == b"" and L.bl_many_config_name(len(shapes)) == b""


def test_struct_layouts_match_the_header(tmp_path):
    # compile the public header with the host C compiler and compare every
    # field's offset and each struct's size with the ctypes mirror in bl.py
    structs = {"bl_options": bl.bl_options, "bl_path": bl.bl_path, "bl_timing": bl.bl_timing}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "biglasso_gpu.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])
