"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/st.h declares (no GPU needed: nothing is called)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "st.h")).read()
    return sorted(set(re.findall(r"\b(st_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ["st_setup", "st_apply", "st_precond", "st_ionic", "st_solve", "st_linsolve",
                 "st_destroy", "st_footprint", "st_wupdate", "st_error_string"]:
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_2311_17500_gb300 import build
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in header_functions():
        assert hasattr(lib, name), name
    from paper_2311_17500_gb300 import _lib
    assert sorted(_lib.EXPORTS) == sorted(n for n in header_functions())


def test_binding_struct_matches_header_field_order():
    from paper_2311_17500_gb300._lib import StProblemDesc
    text = open(os.path.join(ROOT, "include", "st.h")).read()
    body = text[text.index("typedef struct {\n  int d;"):text.index("} st_problem_desc;")]
    fields = re.findall(r"\b(?:int|double|st_stim)\s+([^;]+);", body)
    names = []
    for f in fields:
        for part in f.split(","):
            names.append(re.sub(r"\[.*\]", "", part).strip())
    assert names == [n for n, _ in StProblemDesc._fields_]
