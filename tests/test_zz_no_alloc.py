"""bs_dot_noalloc: the inner product for callers that cannot allocate device
memory (an application that owns every device allocation through its own
pool, or a loop that cannot afford cudaMalloc's device-wide synchronisation).

Calls the entry point through the C ABI twice in a row, on different inputs,
and checks each result against bs_dot within the reductions' 1e-13 relative
tolerance: the second call must not see the first call's leftovers in the
shared static scratch.  This file sorts last so that a stop-at-first-failure
run has already run every other test.
"""
import ctypes

import pytest
import torch

from paper_2009_10917_gb300 import bs, synth

pytestmark = pytest.mark.gpu


def _fn():
    f = bs.lib().bs_dot_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def test_dot_noalloc_matches_bs_dot_on_two_calls_in_a_row():
    f = _fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, seed in [(1234567, 21), (65539, 22)]:
        x = torch.from_numpy(synth.uniform(n, seed, 0)).cuda()
        y = torch.from_numpy(synth.uniform(n, seed, 1)).cuda()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = f(n, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
               ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == bs.BS_OK, bs.lib().bs_last_error()
        want = bs.dot(x, y).cpu().item()
        got = out.cpu().item()
        assert abs(got - want) <= 1e-13 * abs(want)
