"""The element-interior block-Jacobi preconditioner (BS_CG_BLOCK_JACOBI)
against the oracle's block-Jacobi PCG, which factors every interior block
A_II of c_e S_e + lambda M_e by Cholesky (the oracle is pinned against a dense
numpy PCG with the same preconditioner).

The library applies A_II^-1 by fast diagonalisation in float-float arithmetic
(about 2^-46 relative per application) where the oracle uses Cholesky in
FP64; the two differ by rounding, so the r.r histories agree to 1e-5 relative
over the first iterations and the iteration counts to tolerance within
max(3, 2%) (the CG iteration-count bound); the solution satisfies the FP64
true residual bound.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth

pytestmark = pytest.mark.gpu

BJ = bs.BS_CG_BLOCK_JACOBI


def _case(K, N, lam=1e-2, seed=4, masked=0.0):
    m = synth.Mesh(K, N, seed=seed)
    ids = m.ids.copy()
    if masked > 0:
        ids[synth.uniform(ids.size, seed, 9, 0.0, 1.0) < masked] = -1
        keep = np.unique(ids[ids >= 0])
        remap = np.full(m.NG, -1, np.int64)
        remap[keep] = np.arange(keep.size)
        ids = np.where(ids >= 0, remap[np.maximum(ids, 0)], -1).astype(np.int32)
        NG = int(keep.size)
    else:
        NG = m.NG
    coef = synth.lognormal(m.E, 5)
    Z = bs.Map(m.E, N, NG, ids)
    P = bs.Problem(Z, m.h, lam, coef)
    b = synth.uniform(NG, 6)
    return m, ids, NG, coef, Z, P, b


@pytest.mark.parametrize("K,N", [(3, 2), (3, 3), (3, 5), (2, 7), (2, 9)])
@pytest.mark.parametrize("masked", [0.0, 0.02])
def test_block_jacobi_follows_the_oracle(K, N, masked):
    m, ids, NG, coef, Z, P, b = _case(K, N, masked=masked)
    lam = 1e-2
    hist = torch.zeros(3 * 5001, dtype=torch.float64, device="cuda")
    x, info = P.cg(torch.from_numpy(b).cuda(), tol=1e-10, maxit=5000, flags=BJ, hist=hist)
    xo, it, hr = oracle.pcg_block_jacobi(m.E, N, m.h, lam, ids, NG, b, tol=1e-10, maxit=5000,
                                         coef=coef)
    assert info["rc"] == 0
    assert abs(info["iterations"] - it) <= max(3, 0.02 * it), (info["iterations"], it)
    h = hist.cpu().numpy().reshape(-1, 3)
    k = min(8, it, info["iterations"])
    np.testing.assert_allclose(h[:k, 2], hr[1:k + 1], rtol=1e-5)
    r = b - oracle.apply_A(m.E, N, m.h, lam, ids, NG, x.cpu().numpy(), coef)
    assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(b)
    _, itj, _ = oracle.pcg_jacobi(m.E, N, m.h, lam, ids, NG, b, tol=1e-10, maxit=5000, coef=coef)
    if N == 2 or masked > 0:
        # a one-node interior is the diagonal (block Jacobi is Jacobi); with masking,
        # elements with a masked interior node keep Jacobi on their interior
        assert info["iterations"] <= itj + max(3, 0.02 * itj)
    else:
        assert info["iterations"] < itj


@pytest.mark.parametrize("flags", [bs.BS_CG_GRAPH, bs.BS_CG_GRAPH | bs.BS_CG_FF_OPERATOR])
def test_block_jacobi_graph_and_float_float_operator(flags):
    m, ids, NG, coef, Z, P, b = _case(4, 5)
    bt = torch.from_numpy(b).cuda()
    x0, i0 = P.cg(bt, tol=1e-9, maxit=5000, flags=BJ)
    x1, i1 = P.cg(bt, tol=1e-9, maxit=5000, flags=BJ | flags)
    assert i1["rc"] == 0 and abs(i1["iterations"] - i0["iterations"]) <= max(3, 0.02 * i0["iterations"])
    if not flags & bs.BS_CG_FF_OPERATOR:
        assert torch.equal(x0, x1)  # the graph replays the same launches
    r = b - oracle.apply_A(m.E, 5, m.h, 1e-2, ids, NG, x1.cpu().numpy(), coef)
    assert np.linalg.norm(r) <= 2e-9 * np.linalg.norm(b)


def test_block_jacobi_scale_invariance():
    """Per-element power-of-two normalisation: the same steps at any scale."""
    m, ids, NG, coef, Z, P, b = _case(3, 4)
    _, i1 = P.cg(torch.from_numpy(b).cuda(), tol=1e-9, maxit=5000, flags=BJ)
    for sc in (2.0 ** -300, 2.0 ** 300):
        _, i2 = P.cg(torch.from_numpy(b * sc).cuda(), tol=1e-9, maxit=5000, flags=BJ)
        assert i2["rc"] == 0 and i2["iterations"] == i1["iterations"]


def test_block_jacobi_rejections():
    m, ids, NG, coef, Z, P, b = _case(2, 1)
    with pytest.raises(bs.BSError):  # degree 1 has no element interior
        P.cg(torch.from_numpy(b).cuda(), tol=1e-8, flags=BJ)
    m, ids, NG, coef, Z, P, b = _case(2, 3)
    with pytest.raises(bs.BSError):
        P.cg(torch.from_numpy(b).cuda(), tol=1e-8, flags=BJ | bs.BS_CG_SCATTERED)
    mg = synth.Mesh(2, 3, seed=3, perturb=0.1)
    Pg = bs.Problem(bs.Map(mg.E, 3, mg.NG, mg.ids), mg.h, 1.0, verts=mg.verts())
    with pytest.raises(bs.BSError):
        Pg.cg(torch.zeros(mg.NG, dtype=torch.float64, device="cuda") + 1.0, tol=1e-8, flags=BJ)
