"""Operator modes (bs_operator_mode).

The fused operator (BS_OP_FUSED): single-copy nodes written by the element
kernel, shared ones gathered from their own CSR.

A p must be bitwise that of the unfused path -- element kernel plus the
gather of every row -- because a one-copy row's serial sum is +0 + v, which
the fused kernel writes directly.  Checked for the FP64, float-float and
FP32 (inside the refined solver) element kernels, on natural-boundary,
Dirichlet-masked, randomly masked maps and maps with global nodes no local
node references.  CG with the fused p.Ap (summed in another order) follows
the unfused CG to rounding and meets the oracle's residual.

The even-odd element kernels (the default for odd N <= 9) against the direct
sum factorisation (BS_OP_DIRECT) and the oracle: the same 1e-12 max|A p|
bound as the direct kernel (both round every term once; the even-odd form
adds the e/o sums and its tables' rounding, a few units of eps sum |K||u|).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture
def fusion():
    prev = bs.operator_mode(-1)
    yield
    bs.operator_mode(prev)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def both(fn):
    """(fused result, unfused result)."""
    bs.operator_fusion(1)
    a = fn()
    bs.operator_fusion(0)
    b = fn()
    return a, b


def test_fusion_switch(fusion):
    assert bs.operator_mode(-1) == 0  # the default: unfused, even-odd
    assert bs.operator_fusion(-1) == 0
    assert bs.operator_fusion(1) == 0
    assert bs.operator_fusion(-1) == 1
    assert bs.operator_fusion(0) == 1
    assert bs.operator_fusion(7) == 0
    assert bs.operator_fusion(-1) == 1


def _maps():
    out = []
    for K, N in ((1, 1), (2, 2), (3, 3), (4, 5), (3, 7), (2, 8), (1, 12)):
        out.append((f"natural-{K}-{N}", synth.Mesh(K, N, seed=K * N), None))
    for K, N in ((3, 4), (4, 7)):
        out.append((f"dirichlet-{K}-{N}", synth.Mesh(K, N, seed=5, dirichlet=True), None))
    m = synth.Mesh(4, 3, seed=9)
    ids = m.ids.copy()
    ids[synth.uniform(ids.size, 3, 0, 0.0, 1.0) < 0.2] = -1  # random masks: some rows empty
    out.append(("masked-4-3", m, ids))
    m = synth.Mesh(3, 5, seed=2)
    out.append(("unreferenced-3-5", m, "extra"))
    return out


@pytest.mark.parametrize("name,m,ids", _maps(), ids=[t[0] for t in _maps()])
@pytest.mark.parametrize("ff", [False, True])
def test_fused_apply_is_bitwise_unfused(fusion, name, m, ids, ff):
    NG = m.NG
    if isinstance(ids, str):  # five global nodes no local node references
        NG = m.NG + 5
        ids = m.ids
    elif ids is None:
        ids = m.ids
    Z = bs.Map(m.E, m.N, NG, ids)
    coef = synth.lognormal(m.E, 3)
    P = bs.Problem(Z, m.h, 0.4, coef)
    p = cuda(synth.uniform(NG, 4))
    apply = P.apply_A_ff if ff else P.apply_A
    a, b = both(lambda: apply(p, torch.full_like(p, 3.0)).clone())
    assert torch.equal(a, b)
    if NG > m.NG:
        assert bool(torch.all(a[m.NG:] == 0))
    if not ff:
        want = oracle.apply_A(m.E, m.N, m.h, 0.4, ids, NG, p.cpu().numpy(), coef)
        assert np.abs(a.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("flags", [0, bs.BS_CG_JACOBI, bs.BS_CG_FF_OPERATOR,
                                   bs.BS_CG_GRAPH | bs.BS_CG_JACOBI | bs.BS_CG_FF_OPERATOR])
def test_fused_cg_follows_unfused(fusion, flags):
    m = synth.Mesh(6, 5, seed=3)
    Z = bs.Map(m.E, m.N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 1.0)
    bh = synth.uniform(m.NG, 8)
    b = cuda(bh)
    (xa, ia), (xb, ib) = both(lambda: P.cg(b, tol=1e-10, maxit=3000, flags=flags))
    assert abs(ia["iterations"] - ib["iterations"]) <= 1
    assert float(torch.linalg.norm(xa - xb) / torch.linalg.norm(xb)) <= 1e-8
    r = bh - oracle.apply_A(m.E, m.N, m.h, 1.0, m.ids, m.NG, xa.cpu().numpy())
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(bh)


def test_fused_refined_and_learned_follow_unfused(fusion):
    m = synth.Mesh(4, 5, seed=4)
    Z = bs.Map(m.E, m.N, m.NG, m.ids)
    coef = synth.lognormal(m.E, 2)
    P = bs.Problem(Z, m.h, 1e-2, coef)
    bh = synth.uniform(m.NG, 6)
    b = cuda(bh)
    (xa, ia), (xb, ib) = both(lambda: P.cg_refined_f32(b, tol=1e-10, flags=bs.BS_CG_GRAPH))
    assert ia["rel_residual"] <= 1e-10 and ib["rel_residual"] <= 1e-10
    assert abs(ia["iterations"] - ib["iterations"]) <= max(3, ib["iterations"] // 50)
    (xa, ia), (xb, ib) = both(lambda: bs.fpcg_learned(P, None, b, tol=1e-9))
    assert abs(ia["iterations"] - ib["iterations"]) <= 1
    r = bh - oracle.apply_A(m.E, m.N, m.h, 1e-2, m.ids, m.NG, xa.cpu().numpy(), coef=coef)
    assert np.linalg.norm(r) <= 1.5e-9 * np.linalg.norm(bh)


def test_fused_small_config_histories_match_oracle(fusion):
    """50 fixed iterations on the small configuration (K = 8, N = 3): the
    fused p.Ap keeps alpha, beta and r.r within the unfused path's tolerance
    of the oracle."""
    bs.operator_fusion(1)
    m = synth.Mesh(8, 3, seed=1)
    Z = bs.Map(m.E, 3, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 1.0)
    bh = synth.uniform(m.NG, 1, stream=7)
    hist = torch.zeros(3 * 51, dtype=torch.float64, device="cuda")
    x, info = P.cg(cuda(bh), tol=0.0, maxit=50, flags=bs.BS_CG_FIXED_ITERS, hist=hist)
    xo, it, ha, hb, hr = oracle.cg(m.E, 3, m.h, 1.0, m.ids, m.NG, bh, maxit=50, fixed_iters=True)
    h = hist.cpu().numpy()[:150].reshape(50, 3)
    np.testing.assert_allclose(h[:, 0], ha, rtol=1e-10)
    np.testing.assert_allclose(h[:, 1], hb, rtol=1e-10)
    np.testing.assert_allclose(h[:, 2], hr[1:], rtol=1e-10)


@pytest.mark.parametrize("K,N", [(5, 1), (4, 3), (3, 5), (3, 7), (2, 9)])
@pytest.mark.parametrize("fused", [0, bs.BS_OP_FUSED])
def test_evenodd_matches_direct_and_oracle(fusion, K, N, fused):
    m = synth.Mesh(K, N, seed=K + 2 * N)
    coef = synth.lognormal(m.E, 6)
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 0.7, coef)
    p = cuda(synth.uniform(m.NG, 5))
    uL = cuda(synth.uniform(m.NL, 6))
    bs.operator_mode(fused)
    a, aL = P.apply_A(p).clone(), P.apply_local(uL).clone()
    bs.operator_mode(fused | bs.BS_OP_DIRECT)
    d, dL = P.apply_A(p).clone(), P.apply_local(uL).clone()
    want = oracle.apply_A(m.E, N, m.h, 0.7, m.ids, m.NG, p.cpu().numpy(), coef)
    wantL = oracle.apply_local(m.E, N, m.h, 0.7, uL.cpu().numpy(), coef)
    for got in (a, d):
        assert np.abs(got.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()
    for got in (aL, dL):
        assert np.abs(got.cpu().numpy() - wantL).max() <= 1e-12 * np.abs(wantL).max()
    assert not torch.equal(a, d) or N == 1  # the even-odd kernel did run


def test_evenodd_fp32_refined_and_scattered(fusion):
    """The FP32 even-odd kernel inside the refined solver, and the even-odd
    kernel on contiguous local data in scattered-storage CG."""
    m = synth.Mesh(4, 7, seed=2)
    Z = bs.Map(m.E, 7, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 1.0)
    bh = synth.uniform(m.NG, 3)
    b = cuda(bh)
    for flags in (0, bs.BS_CG_SCATTERED):
        x, info = P.cg(b, tol=1e-10, maxit=3000, flags=flags)
        r = bh - oracle.apply_A(m.E, 7, m.h, 1.0, m.ids, m.NG, x.cpu().numpy())
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(bh)
    x, info = P.cg_refined_f32(b, tol=1e-10)
    r = bh - oracle.apply_A(m.E, 7, m.h, 1.0, m.ids, m.NG, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(bh)


def test_fused_on_a_problem_created_under_another_mode(fusion):
    """The fused operator's per-block partials hold one value per element,
    enough for any element-kernel form: a problem made while the direct form
    was selected (4 elements per block at N = 7) runs fused with the
    even-odd form (2 per block)."""
    bs.operator_mode(bs.BS_OP_DIRECT)
    m = synth.Mesh(5, 7, seed=3)
    Z = bs.Map(m.E, 7, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 1.0)
    bs.operator_mode(0)
    bh = synth.uniform(m.NG, 4)
    b = cuda(bh)
    (xa, ia), (xb, ib) = both(lambda: P.cg(b, tol=1e-10, maxit=3000, flags=bs.BS_CG_GRAPH))
    assert abs(ia["iterations"] - ib["iterations"]) <= 1
    r = bh - oracle.apply_A(m.E, 7, m.h, 1.0, m.ids, m.NG, xa.cpu().numpy())
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(bh)
