"""GPU parity of the operator A = Z^T (c S_L + lambda M_L) Z and of CG
(Algorithm 1), against the FP64 oracle, through the C ABI.

Operator tolerance: the GPU contracts with K = D^T W D (one pass), the oracle
takes the gradient then its transpose (two passes); both round every term
once, so each entry differs by at most about (6 Nq) eps sum_j |A_ij p_j|.
For p uniform in [-1, 1) that sum is within a small factor of max|A p|, so
|gpu - oracle| <= 1e-12 max|A p| has two orders of magnitude of margin.
CG: the iterates differ only by reduction order, which finite precision CG
amplifies slowly; after 50 iterations alpha_j, beta_j, r_j.r_j agree to 1e-10
relative and x to 1e-9 (norm-wise) on the small configuration.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth

pytestmark = pytest.mark.gpu


def make(K, N, lam=1.0, coef=None, seed=1):
    m = synth.Mesh(K, N, seed=seed)
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, lam, coef)
    return m, Z, P


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("K,N", [(1, 1), (2, 2), (8, 3), (3, 5), (2, 7), (3, 8), (1, 11), (1, 15)])
@pytest.mark.parametrize("with_coef", [False, True])
def test_apply_A(K, N, with_coef):
    m = synth.Mesh(K, N, seed=K + N)
    coef = synth.lognormal(m.E, 11) if with_coef else None
    lam = 0.3
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, lam, coef)
    p = synth.uniform(m.NG, 12)
    Ap = P.apply_A(cuda(p)).cpu().numpy()
    want = oracle.apply_A(m.E, N, m.h, lam, m.ids, m.NG, p, coef)
    assert np.max(np.abs(Ap - want)) <= 1e-12 * np.max(np.abs(want))
    uL = synth.uniform(m.NL, 13)
    AuL = P.apply_local(cuda(uL)).cpu().numpy()
    wantL = oracle.apply_local(m.E, N, m.h, lam, uL, coef)
    assert np.max(np.abs(AuL - wantL)) <= 1e-12 * np.max(np.abs(wantL))
    d = P.diag().cpu().numpy()
    np.testing.assert_allclose(d, oracle.diag_A(m.E, N, m.h, lam, m.ids, m.NG, coef), rtol=1e-13)


@pytest.mark.parametrize("K,N", [(2, 2), (3, 5), (2, 7), (3, 8)])
@pytest.mark.parametrize("with_coef", [False, True])
def test_apply_A_entrywise(K, N, with_coef):
    """Entry by entry: both sides evaluate the element operator as products
    of 1-D factors (D, W, D^T) and round every product and sum once, so entry
    i of A p is off from the exact value by at most about (2 Nq + 4) eps times
    B_i = (Z^T (c |S|_f + lambda M) Z |p|)_i, where |S|_f is the stiffness
    built from |D|^T W |D| instead of D^T W D (the sizes of the terms that are
    actually summed; numpy's dense Kronecker assembly).  Two such errors
    apart, with a factor two of margin: |gpu - oracle|_i <= 4 (2 Nq + 4) eps B_i
    -- a per-entry form of the max-norm bound of test_apply_A."""
    from tests import fem_ref
    m = synth.Mesh(K, N, seed=K + N)
    coef = synth.lognormal(m.E, 11) if with_coef else np.ones(m.E)
    lam = 0.3
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, lam, coef if with_coef else None)
    p = synth.uniform(m.NG, 12)
    Ap = P.apply_A(cuda(p)).cpu().numpy()
    want = oracle.apply_A(m.E, N, m.h, lam, m.ids, m.NG, p, coef if with_coef else None)
    r, w, D = fem_ref.gll_np(N)
    W = np.diag(w)
    Ka = np.abs(D).T @ W @ np.abs(D)
    kron3 = lambda a, b, c: np.kron(a, np.kron(b, c))
    Sa = 0.5 * m.h * (kron3(W, W, Ka) + kron3(W, Ka, W) + kron3(Ka, W, W))
    Mm = (0.5 * m.h) ** 3 * kron3(W, W, W)
    pa = np.abs(p)[m.ids].reshape(m.E, m.Np)
    wl = (coef[:, None] * (pa @ Sa.T)) + lam * (pa @ Mm.T)
    B = np.zeros(m.NG)
    np.add.at(B, m.ids, wl.reshape(-1))
    eps = np.finfo(np.float64).eps
    bound = 4 * (2 * (N + 1) + 4) * eps * B
    assert np.all(np.abs(Ap - want) <= bound), float(np.max(np.abs(Ap - want) / bound))


def test_operator_annihilates_constants():
    m, Z, P = make(4, 5, lam=0.0)
    one = torch.ones(m.NG, dtype=torch.float64, device="cuda")
    assert float(P.apply_A(one).abs().max()) < 1e-13


@pytest.mark.parametrize("graph", [False, True])
def test_cg_small_config_50_iterations(graph):
    """The small configuration: K=8, N=3, lambda=1, 50 fixed iterations."""
    m, Z, P = make(8, 3, lam=1.0)
    b = synth.uniform(m.NG, 1, stream=7)
    hist = torch.zeros(3 * 51, dtype=torch.float64, device="cuda")
    flags = bs.BS_CG_FIXED_ITERS | (bs.BS_CG_GRAPH if graph else 0)
    x, info = P.cg(cuda(b), tol=0.0, maxit=50, flags=flags, hist=hist)
    assert info["iterations"] == 50 and info["rc"] == 0
    xo, it, al, be, rr = oracle.cg(m.E, 3, m.h, 1.0, m.ids, m.NG, b, maxit=50, fixed_iters=True)
    h = hist.cpu().numpy().reshape(-1, 3)[:50]
    np.testing.assert_allclose(h[:, 0], al, rtol=1e-10)
    np.testing.assert_allclose(h[:, 1], be, rtol=1e-10)
    np.testing.assert_allclose(h[:, 2], rr[1:], rtol=1e-10)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)


def test_cg_graph_matches_plain_bitwise():
    m, Z, P = make(5, 4, lam=1.0, seed=3)
    b = cuda(synth.uniform(m.NG, 2))
    x1, i1 = P.cg(b, tol=1e-9, maxit=500)
    x2, i2 = P.cg(b, tol=1e-9, maxit=500, flags=bs.BS_CG_GRAPH)
    assert i1["iterations"] == i2["iterations"]
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("jacobi", [False, True])
def test_cg_to_tolerance(jacobi):
    coef = synth.lognormal(4 ** 3, 5)
    m, Z, P = make(4, 4, lam=1e-2, coef=coef, seed=4)
    b = synth.uniform(m.NG, 3)
    x, info = P.cg(cuda(b), tol=1e-8, maxit=2000, flags=bs.BS_CG_JACOBI if jacobi else 0)
    assert info["rc"] == 0 and info["rel_residual"] <= 1e-8
    if jacobi:
        xo, it, rr = oracle.pcg_jacobi(m.E, 4, m.h, 1e-2, m.ids, m.NG, b, tol=1e-8, maxit=2000,
                                       coef=coef)
    else:
        xo, it, *_ = oracle.cg(m.E, 4, m.h, 1e-2, m.ids, m.NG, b, tol=1e-8, maxit=2000, coef=coef)
    # iteration counts: the two sides sum the inner products in different
    # orders, and finite-precision CG carries such differences forward (lost
    # orthogonality), so the recursive residual crosses the tolerance a few
    # iterations apart: max(3, 1%) of the oracle's count
    assert abs(info["iterations"] - it) <= max(3, 0.01 * it)
    # true residual of the GPU solution, by the oracle's operator
    r = b - oracle.apply_A(m.E, 4, m.h, 1e-2, m.ids, m.NG, x.cpu().numpy(), coef)
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(b)


def test_cg_initial_guess():
    m, Z, P = make(3, 3)
    b = cuda(synth.uniform(m.NG, 4))
    x, info = P.cg(b, tol=1e-10, maxit=500)
    x2, info2 = P.cg(b, x=x.clone(), tol=1e-10, maxit=500, flags=bs.BS_CG_X0)
    assert info2["iterations"] <= 5 and info2["rc"] == 0


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_cg_breakdown_is_reported(bad):
    """A non-finite right-hand side makes p.Ap non-finite on the first
    iteration: the solve stops with BS_ERR_BREAKDOWN (the fault is injected
    on the host; the GPU stays healthy)."""
    m, Z, P = make(3, 2, lam=1.0)
    b = cuda(synth.uniform(m.NG, 5))
    b[3] = bad
    x, info = P.cg(b, tol=1e-8, maxit=10, check=False)
    assert info["rc"] == bs.BS_ERR_BREAKDOWN
    # the context is still usable
    b = cuda(synth.uniform(m.NG, 5))
    P2 = bs.Problem(Z, m.h, 1.0)
    x, info = P2.cg(b, tol=1e-8, maxit=500)
    assert info["rc"] == 0


def test_cg_not_converged_and_zero_rhs():
    m, Z, P = make(4, 3)
    b = cuda(synth.uniform(m.NG, 6))
    x, info = P.cg(b, tol=1e-14, maxit=3, check=False)
    assert info["rc"] == bs.BS_ERR_NOT_CONVERGED and info["iterations"] == 3
    z = torch.zeros(m.NG, dtype=torch.float64, device="cuda")
    x, info = P.cg(z, tol=1e-8, maxit=10)
    assert info["iterations"] == 0 and float(x.abs().max()) == 0.0
