"""The index predicates of the checked build (-DBS_CHECK=1), compiled from
the same header the kernels include, on the host; and the check entry points
of the default build, which record nothing and need no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2009_10917_gb300", "csrc")

WRAP = r"""
#include "bs_check_pred.h"
int w_index(int64_t i, int64_t n) { return bs_pred_index(i, n); }
int w_map(int64_t id, int64_t ng) { return bs_pred_map_entry(id, ng); }
int w_fused(int64_t c, int64_t ng) { return bs_pred_fused_entry(c, ng); }
int w_row(int64_t a, int64_t b, int64_t nnz) { return bs_pred_row(a, b, nnz); }
int w_tile(int64_t r0, int64_t r1, int64_t k0, int64_t k1, int64_t nr, int64_t nnz, int64_t mx) {
  return bs_pred_tile(r0, r1, k0, k1, nr, nnz, mx);
}
int w_staged(int64_t o, int64_t n) { return bs_pred_staged(o, n); }
"""


@pytest.fixture(scope="module")
def pred(tmp_path_factory):
    d = tmp_path_factory.mktemp("pred")
    src, so = d / "wrap.c", d / "wrap.so"
    src.write_text(WRAP)
    subprocess.run(["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-shared", "-fPIC", "-I", CSRC,
                    str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    i64 = ctypes.c_int64
    for name, n in [("w_index", 2), ("w_map", 2), ("w_fused", 2), ("w_row", 3), ("w_tile", 7),
                    ("w_staged", 2)]:
        f = getattr(L, name)
        f.argtypes = [i64] * n
        f.restype = ctypes.c_int
    return L


def test_index(pred):
    assert [pred.w_index(i, 5) for i in (-1, 0, 4, 5, 6)] == [0, 1, 1, 0, 0]
    assert pred.w_index(0, 0) == 0
    assert pred.w_index(1 << 40, (1 << 40) + 1) == 1
    assert pred.w_index(-(1 << 62), 5) == 0


def test_map_entry(pred):
    # any negative entry masks a node; every other one is a global index < N_G
    assert [pred.w_map(v, 10) for v in (-7, -1, 0, 9, 10, 2**31 - 1)] == [1, 1, 1, 1, 0, 0]
    assert pred.w_map(0, 0) == 0 and pred.w_map(-1, 0) == 1


def test_fused_entry(pred):
    # g (single copy), -1 masked, -2 - g (shared), every g < N_G
    got = [pred.w_fused(c, 10) for c in (9, 10, 0, -1, -2, -11, -12)]
    assert got == [1, 0, 1, 1, 1, 1, 0]


def test_row(pred):
    cases = [((0, 0, 0), 1), ((3, 5, 5), 1), ((2, 1, 5), 0), ((-1, 0, 5), 0), ((3, 6, 5), 0),
             ((5, 5, 5), 1)]
    for args, want in cases:
        assert pred.w_row(*args) == want, args


def test_tile(pred):
    mx = 2048
    ok = [(0, 3, 0, 100, 10, 5000, mx), (0, 1, 0, 5000, 10, 5000, mx), (0, 0, 0, 0, 0, 0, mx),
          (9, 10, 4000, 5000, 10, 5000, mx), (2, 2, 7, 7, 10, 5000, mx)]
    bad = [(0, 2, 0, 5000, 10, 5000, mx),   # two rows over the tile limit
           (0, 11, 0, 10, 10, 5000, mx),    # rows past the CSR
           (0, 1, 0, 5001, 10, 5000, mx),   # entries past the CSR
           (3, 2, 0, 10, 10, 5000, mx),     # decreasing rows
           (0, 1, 10, 9, 10, 5000, mx),     # decreasing entries
           (-1, 1, 0, 9, 10, 5000, mx)]
    assert all(pred.w_tile(*a) == 1 for a in ok)
    assert all(pred.w_tile(*a) == 0 for a in bad)


def test_staged(pred):
    assert [pred.w_staged(o, 6) for o in (-1, 0, 5, 6)] == [0, 1, 1, 0]
    assert pred.w_staged(0, 0) == 0


def test_every_code_is_named_once():
    """Each BS_CHK_* code is distinct and bs_check_device names each one."""
    hdr = open(os.path.join(CSRC, "bs_check_pred.h")).read()
    codes = dict((n, int(v)) for n, v in re.findall(r"(BS_CHK_\w+)\s*=\s*(\d+)", hdr))
    assert len(codes) >= 10 and len(set(codes.values())) == len(codes)
    core = open(os.path.join(CSRC, "bs_core.cu")).read()
    for n in codes:
        assert core.count(f"case {n}:") == 1, n


def test_default_build_records_nothing():
    from paper_2009_10917_gb300 import build
    L = ctypes.CDLL(build.build())
    assert L.bs_check_enabled() == 0
    assert L.bs_check_device() == 0   # returns before any CUDA call
