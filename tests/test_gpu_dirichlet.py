"""Homogeneous Dirichlet problems on the GPU: every solver, on a map whose
boundary copies are masked, converges to the oracle's solution and to the
exact solution of the continuous problem.

-Laplace u = f on the unit cube with u = 0 on its boundary (lambda = 0: the
masked map is what makes A definite), u a sum of three sine modes (not an
eigenvector of A, so CG needs many steps) and f = -Laplace u exactly.  The
load vector uses the collocated GLL mass, b = Z^T M_L Z f.  At N = 7 on 4^3
the discrete solution is within 4.6e-8 of u at the nodes; stopping at a
relative residual of 1e-10 moves the iterate less than 3e-11 from the
converged one (both measured with the oracle), so a GPU solution is accepted
within 1e-9 of the oracle's converged solution and 1e-9 beyond the oracle's
discretisation error.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth
from tests import fem_ref

pytestmark = pytest.mark.gpu

MODES = ((1, 1, 1, 1.0), (2, 3, 1, 0.5), (3, 1, 4, 0.25))


def manufactured(K, N, coef=None):
    m = synth.Mesh(K, N, seed=K + N, dirichlet=True)
    x, y, z = fem_ref.global_coords(m)
    u = np.zeros(m.NG)
    f = np.zeros(m.NG)
    for i, j, k, a in MODES:
        s = a * np.sin(i * np.pi * x) * np.sin(j * np.pi * y) * np.sin(k * np.pi * z)
        u += s
        f += np.pi ** 2 * (i * i + j * j + k * k) * s
    b = oracle.apply_A(m.E, N, m.h, 1.0, m.ids, m.NG, f, coef=np.zeros(m.E))
    uo, _, _, _, _ = oracle.cg(m.E, N, m.h, 0.0, m.ids, m.NG, b, tol=1e-13, maxit=20000,
                               coef=coef)
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 0.0, coef)
    return m, Z, P, b, u, uo


def check(x, b, u, uo, m, slack=1e-9):
    x = x.cpu().numpy() if torch.is_tensor(x) else x
    r = b - oracle.apply_A(m.E, m.N, m.h, 0.0, m.ids, m.NG, x)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
    assert np.abs(x - uo).max() <= slack
    assert np.abs(x - u).max() <= np.abs(uo - u).max() + slack


@pytest.fixture(scope="module")
def n7():
    return manufactured(4, 7)


def test_dirichlet_discretisation_error(n7):
    m, Z, P, b, u, uo = n7
    assert np.abs(uo - u).max() < 1e-7


def test_dirichlet_operator_matches_oracle(n7):
    m, Z, P, b, u, uo = n7
    p = synth.uniform(m.NG, 4)
    Ap = P.apply_A(torch.from_numpy(p).cuda()).cpu().numpy()
    want = oracle.apply_A(m.E, m.N, m.h, 0.0, m.ids, m.NG, p)
    assert np.abs(Ap - want).max() <= 1e-12 * np.abs(want).max()
    d = P.diag().cpu().numpy()
    np.testing.assert_allclose(d, oracle.diag_A(m.E, m.N, m.h, 0.0, m.ids, m.NG), rtol=1e-13)


@pytest.mark.parametrize("flags", [0, bs.BS_CG_GRAPH, bs.BS_CG_JACOBI,
                                   bs.BS_CG_GRAPH | bs.BS_CG_FF_OPERATOR,
                                   bs.BS_CG_JACOBI | bs.BS_CG_FF_OPERATOR])
def test_dirichlet_cg(n7, flags):
    m, Z, P, b, u, uo = n7
    x, info = P.cg(torch.from_numpy(b).cuda(), tol=1e-10, maxit=5000, flags=flags)
    assert info["rc"] == 0
    check(x, b, u, uo, m)


def test_dirichlet_refined_f32(n7):
    m, Z, P, b, u, uo = n7
    x, info = P.cg_refined_f32(torch.from_numpy(b).cuda(), tol=1e-10, flags=bs.BS_CG_GRAPH)
    assert info["rc"] == 0 and info["outer"] >= 1
    check(x, b, u, uo, m)


@pytest.mark.parametrize("flags", [0, bs.BS_CG_FF_OPERATOR, bs.BS_CG_REFINED_F32])
def test_dirichlet_batched(flags):
    cases = [manufactured(K, N) for K, N in ((4, 7), (3, 5), (2, 8), (5, 3))]
    bs_ = [torch.from_numpy(c[3]).cuda() for c in cases]
    xs = [torch.zeros_like(t) for t in bs_]
    rc, infos = bs.solve_batched([c[2] for c in cases], bs_, xs, tol=1e-10, flags=flags)
    assert rc == 0
    for (m, Z, P, b, u, uo), x, info in zip(cases, xs, infos):
        assert info["status"] == 0
        check(x, b, u, uo, m)


def test_dirichlet_learned_fpcg():
    """Flexible PCG with the exact element-interior inverse as the network's
    odd part: on the masked map it reaches the exact solution in fewer
    iterations than Jacobi-PCG (the correction touches element interiors
    only, which the mask never covers)."""
    K, N = 4, 5
    coef = synth.lognormal(K ** 3, 2)
    m, Z, P, b, u, uo = manufactured(K, N, coef)
    S, M = fem_ref.element_matrices(N, m.h)
    Ae = S  # lambda = 0, c = 1
    Np, n = m.Np, N - 1
    I = np.array([i + (N + 1) * (j + (N + 1) * k) for k in range(1, N) for j in range(1, N)
                  for i in range(1, N)])
    Mint = np.zeros((Np, Np))
    Mint[np.ix_(I, I)] = np.linalg.solve(Ae[np.ix_(I, I)], np.diag(np.diag(Ae)[I])) - np.eye(n ** 3)
    H = 224
    W1 = np.zeros((H, Np), np.float32)
    W1[:Np] = np.eye(Np)
    W2 = np.zeros((Np, H), np.float32)
    W2[:, :Np] = 2 * Mint
    net = bs.MLP(W1, W2, split=True)
    bt = torch.from_numpy(b).cuda()
    x, info = bs.fpcg_learned(P, net, bt, tol=1e-10, flags=bs.BS_FPCG_ODD)
    xj, ij = bs.fpcg_learned(P, None, bt, tol=1e-10)
    assert info["rc"] == 0 and info["outer"] == 0 and ij["rc"] == 0
    assert info["iterations"] < 0.85 * ij["iterations"]
    r = b - oracle.apply_A(m.E, N, m.h, 0.0, m.ids, m.NG, x.cpu().numpy(), coef=coef)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
    # the coefficient changes the solution; the oracle's converged one is the target
    assert np.abs(x.cpu().numpy() - uo).max() <= 1e-9 * np.abs(uo).max()
