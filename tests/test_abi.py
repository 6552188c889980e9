"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/biglasso_gpu.h declares.  No compute call is made (no GPU needed):
only entry points that fail argument checks on the host before touching CUDA."""
import ctypes as C
import os
import re

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


def test_struct_layouts_match_the_header():
    # bl_options: 3 doubles + int64 + 2 int32
    assert C.sizeof(bl.bl_options) == 40
    # bl_path: 15 pointer/int64 fields + lambda_max, jstar, ybar
    assert C.sizeof(bl.bl_path) == 18 * 8
    assert C.sizeof(bl.bl_timing) == 12 * 8 * 3 + 16
