"""GPU parity of the float-float element operator (bs_apply_A_ff) and of CG
run with it (BS_CG_FF_OPERATOR) against the FP64 oracle.

Bound: every input is split into a float pair with relative error 2^-48,
each product of high parts is exact, the cross terms carry a float's 2^-24
of a 2^-24-sized quantity and TwoSum keeps the high sums exact, so a node's
error is a small multiple of 2^-46 (|A| |u|)_node, where |A| is the operator
with every coefficient replaced by its magnitude.  The tests allow 2^-42
(|A| |u|) elementwise, with |A| assembled densely by the independent numpy
reference.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth
from tests import fem_ref

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture
def mode():
    prev = bs.operator_mode(-1)
    yield bs.operator_mode
    bs.operator_mode(prev)


@pytest.mark.parametrize("K,N", [(2, 1), (2, 2), (2, 3), (2, 5), (1, 7), (1, 9)])
@pytest.mark.parametrize("with_coef", [False, True])
@pytest.mark.parametrize("direct", [False, True])
def test_apply_A_ff_within_bound(mode, K, N, with_coef, direct):
    """Both element-kernel forms (even-odd for odd N, the default, and
    direct) of both operators stay within the bound."""
    mode(bs.BS_OP_DIRECT if direct else 0)
    m = synth.Mesh(K, N, seed=3)
    lam = 1e-2
    coef = synth.lognormal(m.E, 5) if with_coef else None
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, lam, coef)
    for scale in (1.0, 1e-20, 1e20):
        u = synth.uniform(m.NG, 7) * scale
        got = P.apply_A_ff(cuda(u)).cpu().numpy()
        want = oracle.apply_A(m.E, N, m.h, lam, m.ids, m.NG, u, coef)
        A = fem_ref.assemble(m, lam, coef)
        bound = np.abs(A) @ np.abs(u)
        assert np.all(np.abs(got - want) <= 2.0 ** -42 * bound)
        # the FP64 operator, for scale: its one-pass K = D^T W D form and the
        # oracle's two passes (gradient, then D^T) differ by rounding of
        # intermediates larger than |A| |u|, a few units of 2^-52 of it
        g64 = P.apply_A(cuda(u)).cpu().numpy()
        assert np.all(np.abs(g64 - want) <= 2.0 ** -46 * bound)


def test_apply_A_ff_tiny_and_zero_inputs():
    """Zero maps to zero; inputs below 2^-102 count as zero (documented);
    inputs of 2^-80 are still inside the split's window."""
    m = synth.Mesh(2, 3, seed=1)
    Z = bs.Map(m.E, 3, m.NG, m.ids)
    P = bs.Problem(Z, m.h, 1.0)
    z = torch.zeros(m.NG, dtype=torch.float64, device="cuda")
    assert float(P.apply_A_ff(z).abs().max()) == 0.0
    tiny = torch.full((m.NG,), 2.0 ** -110, dtype=torch.float64, device="cuda")
    assert float(P.apply_A_ff(tiny).abs().max()) == 0.0
    u = cuda(synth.uniform(m.NG, 4) * 2.0 ** -80)
    got, want = P.apply_A_ff(u), P.apply_A(u)
    assert float((got - want).abs().max()) <= 1e-12 * float(want.abs().max())


@pytest.mark.parametrize("jacobi", [False, True])
def test_cg_with_ff_operator(jacobi):
    N, K, lam = 5, 6, 1e-2
    m = synth.Mesh(K, N, seed=2)
    coef = synth.lognormal(m.E, 3)
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, lam, coef)
    bh = synth.uniform(m.NG, 11)
    b = cuda(bh)
    base = bs.BS_CG_GRAPH | (bs.BS_CG_JACOBI if jacobi else 0)
    x, info = P.cg(b, tol=1e-8, maxit=20000, flags=base | bs.BS_CG_FF_OPERATOR)
    x64, i64 = P.cg(b, tol=1e-8, maxit=20000, flags=base)
    assert info["rc"] == 0
    assert abs(info["iterations"] - i64["iterations"]) <= max(3, 0.02 * i64["iterations"])
    r = bh - oracle.apply_A(m.E, N, m.h, lam, m.ids, m.NG, x.cpu().numpy(), coef)
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(bh)
    assert torch.linalg.norm(x - x64) <= 1e-6 * torch.linalg.norm(x64)


def test_ff_cg_is_scale_invariant():
    """CG with the float-float operator runs the system scaled by the power
    of two that brings b's RMS near 1 and unscales x (exact), so a right-hand
    side of 2^-110 or 2^100 takes the same steps; the hist-free info reports
    the unscaled r.r and b.b."""
    N, K, lam = 3, 4, 1e-2
    m = synth.Mesh(K, N, seed=2)
    Z = bs.Map(m.E, N, m.NG, m.ids)
    P = bs.Problem(Z, m.h, lam)
    b = cuda(synth.uniform(m.NG, 11))
    x1, i1 = P.cg(b, tol=1e-9, maxit=5000, flags=bs.BS_CG_FF_OPERATOR)
    for sc in (2.0 ** -110, 2.0 ** 100):
        xs, is_ = P.cg(b * sc, tol=1e-9, maxit=5000, flags=bs.BS_CG_FF_OPERATOR)
        assert is_["rc"] == 0 and is_["iterations"] == i1["iterations"]
        assert torch.equal(xs / sc, x1)
        assert is_["bb"] == pytest.approx(i1["bb"] * sc * sc, rel=1e-12)
    # an initial guess is scaled with b
    x0 = x1.clone() * 0.5
    xg, ig = P.cg(b * 2.0 ** -110, x=x0 * 2.0 ** -110, tol=1e-9, maxit=5000,
                  flags=bs.BS_CG_FF_OPERATOR | bs.BS_CG_X0)
    assert ig["rc"] == 0
    assert torch.linalg.norm(xg / 2.0 ** -110 - x1) <= 1e-7 * torch.linalg.norm(x1)
