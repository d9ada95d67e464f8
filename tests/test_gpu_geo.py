"""General (perturbed) hexahedra on the GPU (bs_problem_create_geo) against
the oracle's general-geometry route (tests/test_oracle_pins.py pins it:
affine case, exact linear fields and volume, rigid-motion invariance).

Operator bound: both sides round every term of the same sums once, in
different orders and with separately rounded geometric factors, so each
entry differs by a few units of eps times sum |A_ij p_j|, well inside
1e-12 max|A p|.  CG: the same 1e-10 history tolerance as the affine
solver's small-configuration test; solves to tolerance meet the oracle's
true residual in the oracle's iteration count (within 2 or 1%).  The CG
cases carry no coefficient: with lognormal coefficients on these small
perturbed meshes a 1e-15 change of b already moves the oracle's own
50-iteration history by O(1) (measured), so histories are compared where
they are stable (1e-15 there).
"""
import functools

import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth
from tests import fem_ref

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make(K, N, lam=0.5, delta=0.2, coef=True, seed=3, dirichlet=False):
    m = synth.Mesh(K, N, seed=seed, perturb=delta, dirichlet=dirichlet)
    c = synth.lognormal(m.E, 4) if coef else None
    V = m.verts()
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, lam, c, verts=V)
    return m, Z, P, c, V


@pytest.mark.parametrize("K,N", [(3, 1), (3, 3), (2, 4), (2, 7), (1, 11)])
def test_geo_apply_matches_oracle(K, N):
    m, Z, P, c, V = make(K, N)
    p = synth.uniform(m.NG, 5)
    got = P.apply_A(cuda(p)).cpu().numpy()
    want = oracle.apply_A_geo(m.E, N, 0.5, V, m.ids, m.NG, p, c)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    uL = synth.uniform(m.NL, 6)
    gotL = P.apply_local(cuda(uL)).cpu().numpy()
    wantL = oracle.apply_local_geo(m.E, N, 0.5, V, uL, c)
    assert np.abs(gotL - wantL).max() <= 1e-12 * np.abs(wantL).max()
    d = P.diag().cpu().numpy()
    np.testing.assert_allclose(d, oracle.diag_A_geo(m.E, N, 0.5, V, m.ids, m.NG, c), rtol=1e-12)


@pytest.mark.parametrize("K,N", [(3, 1), (3, 3), (2, 4), (2, 7), (1, 11)])
def test_geo_float_float_apply_matches_oracle(K, N):
    """The float-float general-geometry kernel: every value a float pair
    (about 2^-46 relative per term), so within 1e-11 max|A p| of the oracle,
    at unit scale and scaled by 2^-60 (its inputs stay inside the float-pair
    window)."""
    m, Z, P, c, V = make(K, N)
    for scale in (1.0, 2.0 ** -60):
        p = synth.uniform(m.NG, 5) * scale
        got = P.apply_A_ff(cuda(p)).cpu().numpy()
        want = oracle.apply_A_geo(m.E, N, 0.5, V, m.ids, m.NG, p, c)
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("shrink", [2.0 ** -20, 2.0 ** -28])
def test_geo_float_float_on_a_small_domain(shrink):
    """The geometric factors themselves scale with the mesh: G ~ w h / 2 and
    lambda w det J ~ lambda h^3.  On a domain shrunk by 2^-20 and by 2^-28
    (stiffness factors near 2^-30, all inside the float-pair window that
    starts at 2^-102) the float-float kernel still agrees with the oracle
    within 1e-11 max|A p|.  (The mass term then lies below the stiffness
    term's rounding on both sides, so A p is the stiffness part.)"""
    m = synth.Mesh(2, 4, seed=3, perturb=0.2)
    c = synth.lognormal(m.E, 4)
    V = m.verts() * shrink
    Z = bs.Map(m.E, 4, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 0.5, c, verts=V)
    p = synth.uniform(m.NG, 5)
    got = P.apply_A_ff(cuda(p)).cpu().numpy()
    want = oracle.apply_A_geo(m.E, 4, 0.5, V, m.ids, m.NG, p, c)
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


def test_geo_on_cubes_matches_the_affine_problem():
    m, Z, P, c, V = make(3, 5, delta=0.0)
    Pa = bs.Problem(Z, m.h, 0.5, c)
    p = cuda(synth.uniform(m.NG, 7))
    a, g = Pa.apply_A(p), P.apply_A(p)
    assert float((a - g).abs().max()) <= 1e-12 * float(a.abs().max())


@pytest.mark.parametrize("graph", [False, True])
def test_geo_cg_histories_match_oracle(graph):
    m, Z, P, c, V = make(4, 3, lam=1.0, coef=False)
    b = synth.uniform(m.NG, 1, stream=7)
    hist = torch.zeros(3 * 51, dtype=torch.float64, device="cuda")
    flags = bs.BS_CG_FIXED_ITERS | (bs.BS_CG_GRAPH if graph else 0)
    x, info = P.cg(cuda(b), tol=0.0, maxit=50, flags=flags, hist=hist)
    xo, it, al, be, rr = oracle.cg_geo(m.E, 3, 1.0, V, m.ids, m.NG, b, maxit=50,
                                       fixed_iters=True, coef=c)
    h = hist.cpu().numpy().reshape(-1, 3)[:50]
    np.testing.assert_allclose(h[:, 0], al, rtol=1e-10)
    np.testing.assert_allclose(h[:, 1], be, rtol=1e-10)
    np.testing.assert_allclose(h[:, 2], rr[1:], rtol=1e-10)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)


@functools.lru_cache(maxsize=None)
def _oracle_iterations(jacobi):
    m, Z, P, c, V = make(4, 5, coef=False)
    bh = synth.uniform(m.NG, 2)
    if jacobi:
        return oracle.pcg_jacobi_geo(m.E, 5, 0.5, V, m.ids, m.NG, bh, tol=1e-10, maxit=5000,
                                     coef=c)[1]
    return oracle.cg_geo(m.E, 5, 0.5, V, m.ids, m.NG, bh, tol=1e-10, maxit=5000, coef=c)[1]


@pytest.mark.parametrize("flags", [0, bs.BS_CG_GRAPH, bs.BS_CG_JACOBI, bs.BS_CG_SCATTERED,
                                   bs.BS_CG_JACOBI | bs.BS_CG_SCATTERED | bs.BS_CG_GRAPH,
                                   bs.BS_CG_FF_OPERATOR | bs.BS_CG_GRAPH,
                                   bs.BS_CG_FF_OPERATOR | bs.BS_CG_JACOBI | bs.BS_CG_SCATTERED])
def test_geo_cg_to_tolerance(flags):
    m, Z, P, c, V = make(4, 5, coef=False)
    bh = synth.uniform(m.NG, 2)
    x, info = P.cg(cuda(bh), tol=1e-10, maxit=5000, flags=flags)
    assert info["rc"] == 0
    r = bh - oracle.apply_A_geo(m.E, 5, 0.5, V, m.ids, m.NG, x.cpu().numpy(), c)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(bh)
    it = _oracle_iterations(bool(flags & bs.BS_CG_JACOBI))
    assert abs(info["iterations"] - it) <= max(2, it // 100)


def test_geo_manufactured_solution():
    """-Laplace u = f, u = 0 on the boundary of the unit cube meshed by
    perturbed hexahedra (N = 7 on 4^3): the GPU solution is the oracle's
    converged one and within the discretisation error of u."""
    m, Z, P, c, V = make(4, 7, lam=0.0, coef=False, dirichlet=True, seed=1)
    x, y, z = fem_ref.node_coords(m)
    u = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    b = oracle.apply_A_geo(m.E, 7, 1.0, V, m.ids, m.NG, 3 * np.pi ** 2 * u, coef=np.zeros(m.E))
    uo, _, _, _, _ = oracle.cg_geo(m.E, 7, 0.0, V, m.ids, m.NG, b, tol=1e-13, maxit=5000)
    xg, info = P.cg(cuda(b), tol=1e-11, maxit=5000, flags=bs.BS_CG_GRAPH)
    xg = xg.cpu().numpy()
    assert np.abs(xg - uo).max() <= 1e-8
    assert np.abs(uo - u).max() < 1e-5
    assert np.abs(xg - u).max() <= np.abs(uo - u).max() + 1e-8


def test_geo_rejections():
    m, Z, P, c, V = make(2, 3)
    b = cuda(synth.uniform(m.NG, 1))
    with pytest.raises(bs.BSError):
        P.cg_refined_f32(b)
    with pytest.raises(bs.BSError):
        bs.solve_batched([P], [b], [torch.zeros_like(b)])
    with pytest.raises(bs.BSError):
        bs.fpcg_learned(P, None, b)
    bad = V.copy()
    bad[0, [0, 1]] = bad[0, [1, 0]]  # a mirrored element: det J < 0
    with pytest.raises(bs.BSError):
        bs.Problem(Z, m.h, 0.5, c, verts=bad)
    with pytest.raises(bs.BSError):
        m12 = synth.Mesh(1, 12, seed=1)
        bs.Problem(bs.Map(m12.E, 12, m12.NG, m12.ids), m12.h, 1.0, verts=m12.verts())
