"""Bounded device-side waits run out without a fault or a hang.

The batched solver's cooperative kernel separates its phases by grid
barriers whose spins are bounded by a clock budget (bs_set_wait_budget).
With a budget of one cycle every block that is not the last to arrive gives
up at once: the kernel records BS_ERR_TIMEOUT and returns, the blocks that
had passed a barrier give up at the next one, and the call reports the
timeout instead of waiting.  The test then restores the default budget and
checks that the same solves, on the same context, converge and match the
oracle -- the context stays usable and no barrier state leaks between calls.
Graph replay takes the budget from device memory, so it is covered too.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth

pytestmark = pytest.mark.gpu


def _cases():
    out = []
    for i, (N, K) in enumerate([(3, 4), (5, 3), (2, 6), (7, 2)]):
        m = synth.Mesh(K, N, seed=900 + i)
        Z = bs.Map(m.E, N, m.NG, m.ids)
        P = bs.Problem(Z, m.h, 1.0)
        out.append((m, Z, P, synth.uniform(m.NG, 900 + i, stream=3)))
    return out


@pytest.mark.parametrize("flags", [0, bs.BS_CG_GRAPH, bs.BS_CG_GRAPH | bs.BS_CG_REFINED_F32])
def test_batched_barrier_budget_runs_out_then_recovers(flags):
    cases = _cases()
    bs_ = [torch.from_numpy(c[3]).cuda() for c in cases]
    xs = [torch.zeros_like(b) for b in bs_]
    probs = [c[2] for c in cases]
    default = bs.set_wait_budget(1)
    try:
        rc, infos = bs.solve_batched(probs, bs_, xs, tol=1e-8, flags=flags, check=False)
        torch.cuda.synchronize()  # every block has exited: the call returned
    finally:
        assert bs.set_wait_budget(0) == 1
    assert rc == bs.BS_ERR_TIMEOUT
    assert all(i["status"] == bs.BS_ERR_TIMEOUT for i in infos)
    assert default == 1 << 32
    assert bs.set_wait_budget(0) == 1 << 32  # the default is back
    # the same solves on the same context, default budget
    rc, infos = bs.solve_batched(probs, bs_, xs, tol=1e-8, flags=flags, check=False)
    assert rc == bs.BS_OK
    for (m, Z, P, b), info, x in zip(cases, infos, xs):
        assert info["status"] == 0
        r = b - oracle.apply_A(m.E, m.N, m.h, 1.0, m.ids, m.NG, x.cpu().numpy())
        assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(b)
