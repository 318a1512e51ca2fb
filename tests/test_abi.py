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
            names.append(re.sub(r"\[.*\]", "", part).strip().lstrip("*").strip())
    assert names == [n for n, _ in StProblemDesc._fields_]


def test_footprint_validates_and_grows():
    """st_footprint is pure host logic: it rejects invalid descriptions with
    ST_ERR_ARG and grows with every size that allocates (no GPU needed)."""
    import workloads as W
    from paper_2311_17500_gb300 import _lib as L
    from paper_2311_17500_gb300 import build
    build.build()
    base = W.config("c1_newton_2d")
    fp = L.footprint(base)
    assert fp > 0
    four_d = dict(d=4, n_el=[16] * 4, D=[1e-3] * 4,
                  source=dict(kind="stim", boxes=[W.stim_box([0] * 4, [0.1] * 4, 0, 1, 1)]))
    for bad in (dict(p=0), dict(p=5), four_d, dict(n_el=[0, 16]), dict(n_el_t=0), dict(T=-1.0),
                dict(D=[0.0, 1e-3]), dict(gmres_m=0), dict(gmres_m=501), dict(rtol=0.0), dict(alpha=1.5),
                dict(max_fp=0), dict(eps_theta=-0.1)):
        desc = dict(base, **bad)
        with pytest.raises(L.StError) as e:
            L.footprint(desc)
        assert e.value.code == L.ST_ERR_ARG, bad
    for grow in (dict(n_el_t=64), dict(n_el=[32, 16]), dict(n_el=[16, 32]), dict(gmres_m=200), dict(p=3)):
        assert L.footprint(dict(base, **grow)) > fp, grow
    assert L.footprint(dict(base, precision="fp64")) > L.footprint(dict(base, precision="mixed"))
