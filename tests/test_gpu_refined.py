"""GPU parity of the mixed-precision solve: FP32-storage CG inside FP64
iterative refinement, against the FP64 oracle.

The refined solve is judged the way it stops: by the FP64 true residual
||b - A x|| / ||b||, recomputed here with the oracle's operator.  Its x is
compared with the FP64 oracle's CG solution (tol 1e-12); the gap is bounded by
cond(A) times the residual tolerance, and cond(A) stays below 1e3 on these
small meshes.  The outer step count is compared with the oracle's FP32
iterative refinement (the same algorithm in float on the CPU): within one.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K,N,lam,with_coef", [(4, 3, 1.0, False), (8, 3, 1.0, False),
                                               (3, 7, 1.0, False), (4, 5, 1e-2, True)])
@pytest.mark.parametrize("graph", [False, True])
def test_refined_reaches_fp64_tolerance(K, N, lam, with_coef, graph):
    m = synth.Mesh(K, N, seed=K + 10 * N)
    coef = synth.lognormal(m.E, 3) if with_coef else None
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, lam, coef)
    b = synth.uniform(m.NG, 5)
    x, info = P.cg_refined_f32(torch.from_numpy(b).cuda(), tol=1e-10,
                               flags=bs.BS_CG_GRAPH if graph else 0)
    assert info["rc"] == 0 and info["rel_residual"] <= 1e-10
    xg = x.cpu().numpy()
    r = b - oracle.apply_A(m.E, N, m.h, lam, m.ids, m.NG, xg, coef)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
    xo, it, *_ = oracle.cg(m.E, N, m.h, lam, m.ids, m.NG, b, tol=1e-12, maxit=20000, coef=coef)
    assert np.linalg.norm(xg - xo) <= 1e3 * 1e-10 * np.linalg.norm(xo)
    assert info["outer"] >= 2  # FP32 alone cannot reach 1e-10
    _, inner, outer, rel = oracle.cg_ir_f32(m.E, N, m.h, lam, m.ids, m.NG, b, 1e-10, coef=coef)
    assert rel <= 1e-10
    assert abs(info["outer"] - outer) <= 1


def test_refined_initial_guess_and_zero_rhs():
    m = synth.Mesh(4, 4, seed=2)
    Z = bs.Map(m.E, 4, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 1.0)
    b = torch.from_numpy(synth.uniform(m.NG, 6)).cuda()
    x, info = P.cg(b, tol=1e-12, maxit=5000)
    x2, info2 = P.cg_refined_f32(b, x=x.clone(), tol=1e-10, flags=bs.BS_CG_X0)
    assert info2["outer"] == 0 and info2["iterations"] == 0
    z = torch.zeros_like(b)
    x3, info3 = P.cg_refined_f32(z, tol=1e-10)
    assert info3["outer"] == 0 and float(x3.abs().max()) == 0.0


def test_refined_breakdown_on_nan():
    m = synth.Mesh(3, 3, seed=2)
    Z = bs.Map(m.E, 3, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 1.0)
    b = torch.from_numpy(synth.uniform(m.NG, 6)).cuda()
    b[5] = float("nan")
    x, info = P.cg_refined_f32(b, tol=1e-10, check=False)
    assert info["rc"] == bs.BS_ERR_BREAKDOWN
