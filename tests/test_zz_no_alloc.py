"""bs_dot_noalloc: the inner product for callers that cannot allocate device
memory (an application that owns every device allocation through its own
pool, or a loop that cannot afford cudaMalloc's device-wide synchronisation).

Calls the entry point through the C ABI several times in a row, on different
inputs, and checks each result bitwise against bs_dot (the same kernel and,
on a GPU with fewer resident blocks than the static scratch holds, the same
grid and combine order) and within the reductions' 1e-13 relative tolerance
against the oracle's Dot2 sum: a call must not see the previous call's
leftovers in the shared static scratch.  The cases cover the 16-byte vector
path, a common misalignment (scalar head and tail), operands of different
alignment (scalar-only path) and n = 0 (one block writes +0.0) followed by a
normal call.  This file sorts last so that a stop-at-first-failure run has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth

pytestmark = pytest.mark.gpu


def _fn():
    f = bs.lib().bs_dot_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def _operands(n, seed, shift_x, shift_y):
    """x, y of length n as views `shift` elements into longer device buffers,
    and their host values."""
    xh, yh = synth.uniform(n, seed, 0), synth.uniform(n, seed, 1)
    xb = torch.zeros(n + 2, dtype=torch.float64, device="cuda")
    yb = torch.zeros(n + 2, dtype=torch.float64, device="cuda")
    x, y = xb[shift_x:shift_x + n], yb[shift_y:shift_y + n]
    x.copy_(torch.from_numpy(xh))
    y.copy_(torch.from_numpy(yh))
    return x, y, xh, yh


# (n, seed, shift of x, shift of y): aligned, both shifted by one element
# (scalar head and tail around the vector body), different alignments
# (scalar path only), empty, and a normal call after the empty one
CASES = [(1234567, 21, 0, 0), (65539, 22, 1, 1), (300001, 23, 1, 0), (0, 24, 0, 0),
         (4099, 25, 0, 0)]


def test_dot_noalloc_matches_bs_dot_and_the_oracle_on_calls_in_a_row():
    f = _fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, seed, sx, sy in CASES:
        x, y, xh, yh = _operands(n, seed, sx, sy)
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = f(n, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
               ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == bs.BS_OK, bs.lib().bs_last_error()
        got = out.cpu().numpy()
        want = bs.dot(x, y).cpu().numpy()
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (n, got, want)
        o = oracle.dot(xh, yh)
        if n == 0:
            assert got[0] == 0.0 and not np.signbit(got[0])
        else:
            assert abs(got[0] - o) <= 1e-13 * abs(o)


def test_dot_noalloc_argument_errors():
    f = _fn()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert f(-1, None, None, ctypes.c_void_p(out.data_ptr()), None) == bs.BS_ERR_ARG
    assert f(8, None, None, ctypes.c_void_p(out.data_ptr()), None) == bs.BS_ERR_ARG
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert f(8, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None,
             None) == bs.BS_ERR_ARG
