"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/bs.h declares.  No compute calls: this runs without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bs_copy", "bs_axpy", "bs_norm", "bs_dot", "bs_cg_update", "bs_scatter",
                     "bs_gather", "bs_cg_solve", "bs_map_create", "bs_problem_create"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2009_10917_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s+(\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(path)  # loads without a GPU
    for n in declared_functions():
        assert hasattr(L, n)
    L.bs_error_string.restype = ctypes.c_char_p
    assert L.bs_error_string(0) == b"success"
    assert L.bs_version() >= 10000


def test_argument_errors_without_gpu():
    """Argument validation happens before any CUDA call."""
    from paper_2009_10917_gb300 import build
    L = ctypes.CDLL(build.build())
    L.bs_copy.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert L.bs_copy(-1, None, None, None) == 1   # BS_ERR_ARG
    assert L.bs_copy(0, None, None, None) == 0    # empty is valid
    assert L.bs_copy(4, None, None, None) == 1
    L.bs_last_error.restype = ctypes.c_char_p
    assert b"NULL" in L.bs_last_error()


def test_header_constants_match_the_binding():
    """Every BS_* enum value of include/bs.h that the Python binding names
    has the same value there."""
    from paper_2009_10917_gb300 import bs
    text = open(os.path.join(ROOT, "include", "bs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"\b(BS_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    named = [k for k in consts if hasattr(bs, k)]
    assert len(named) >= 20
    for k in named:
        assert getattr(bs, k) == consts[k], k
    for k in ("BS_CG_SCATTERED", "BS_OP_FUSED", "BS_OP_DIRECT", "BS_CG_FF_OPERATOR"):
        assert k in named


def test_operator_mode_and_geometry_arguments_without_gpu():
    """The operator-mode switch is host state; bs_problem_create_geo
    validates its arguments before any CUDA call."""
    from paper_2009_10917_gb300 import build
    L = ctypes.CDLL(build.build())
    L.bs_operator_mode.argtypes = [ctypes.c_int32]
    assert L.bs_operator_mode(-1) == 0          # default: unfused, even-odd
    assert L.bs_operator_mode(3) == 0           # fused | direct
    assert L.bs_operator_mode(-1) == 3
    assert L.bs_operator_mode(0) == 3
    L.bs_problem_create_geo.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert L.bs_problem_create_geo(None, 1.0, None, None, ctypes.byref(out)) == 1
    assert L.bs_problem_create_geo(None, 1.0, None, None, None) == 1
