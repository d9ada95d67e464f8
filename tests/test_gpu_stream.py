"""GPU parity of BS1-BS5 (Table 1) against the FP64 oracle, through the C ABI.

Bitwise: copy, AXPY, the x and r of the fused CG update (explicit fma on both
sides).  Reductions (norm, dot, the r.r of BS5): |gpu - oracle| <= 1e-13 |oracle|.
The oracle's Dot2 is within an ulp of the exact sum; the GPU's grid-stride
plus tree order has an error of about n_thread * eps * sum|x_i y_i| / |x.y|
relative (n_thread <= a few thousand terms per thread), far inside 1e-13 for
these uniform[-1, 1) inputs.
FP32 twins: copy/AXPY/update bitwise against the float oracle; reductions
carried as float pairs, bound 2^-40 * sum |x_i y_i| (float-pair accumulation
keeps ~44-48 bits; 2^-40 leaves margin for the per-thread serial chains).
Sizes span several grid sweeps with ragged tails; offsets 0/1 element cover
the aligned 128-bit path, the scalar head and the mixed-alignment scalar path.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 2, 3, 7, 1000, 65539, 1234567]


def dev(a, off=0):
    """Device copy of a, starting `off` elements into a fresh buffer."""
    t = torch.empty(a.size + off, dtype=torch.from_numpy(a[:0]).dtype, device="cuda")
    t[off:] = torch.from_numpy(a).cuda()
    return t[off:]


def host(t):
    return t.cpu().numpy()


def bits(a):
    return np.ascontiguousarray(a).view(np.uint64 if a.dtype == np.float64 else np.uint32)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("ox,oy", [(0, 0), (1, 1), (0, 1)])
def test_copy_bitwise(n, ox, oy):
    x = synth.uniform(n, 1)
    y = dev(np.full(n, 7.0), oy)
    bs.copy(dev(x, ox), y)
    assert np.array_equal(bits(host(y)), bits(oracle.copy(x)))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("beta", [1.0, 0.0, -0.25])
@pytest.mark.parametrize("ox,oy", [(0, 0), (1, 1), (1, 0)])
def test_axpy_bitwise(n, beta, ox, oy):
    x, y = synth.uniform(n, 2, 0), synth.uniform(n, 2, 1)
    yd = dev(y, oy)
    bs.axpy(0.5 if beta == 1.0 else -1.3, dev(x, ox), beta, yd)
    want = oracle.axpy(0.5 if beta == 1.0 else -1.3, x, beta, y)
    assert np.array_equal(bits(host(yd)), bits(want))


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("off", [0, 1])
def test_norm_dot(n, off):
    x, y = synth.uniform(n, 3, 0), synth.uniform(n, 3, 1)
    xd, yd = dev(x, off), dev(y, off)
    nr = host(bs.norm(xd))
    s, sq = oracle.norm(x)
    if n == 0:
        assert nr[0] == 0.0 and nr[1] == 0.0
    else:
        assert rel(nr[0], s) <= 1e-13 and rel(nr[1], sq) <= 1e-13
    d = host(bs.dot(xd, yd))[0]
    o = oracle.dot(x, y)
    assert abs(d - o) <= 1e-13 * abs(o) + (1e-300 if n else 0.0)
    # deterministic: same grid, same order, same bits
    assert host(bs.dot(xd, yd))[0] == d
    assert np.array_equal(host(bs.norm(xd)), nr)


def test_dot_of_x_with_itself_is_norm_squared():
    x = synth.uniform(300001, 4)
    xd = dev(x)
    d = host(bs.dot(xd, xd))[0]
    s = host(bs.norm(xd))[0]
    assert rel(d, s) <= 2e-16 * 4


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("off", [0, 1])
def test_cg_update(n, off):
    p, Ap, x, r = (synth.uniform(n, 5, s) for s in range(4))
    xd, rd = dev(x, off), dev(r, off)
    rr = host(bs.cg_update(0.37, dev(p, off), dev(Ap, off), xd, rd))[0]
    xo, ro, rro = oracle.cg_update(0.37, p, Ap, x, r)
    assert np.array_equal(bits(host(xd)), bits(xo))
    assert np.array_equal(bits(host(rd)), bits(ro))
    assert (rr == 0.0) if n == 0 else rel(rr, rro) <= 1e-13


# ---------------------------------------------------------------- FP32 twins

@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("off", [0, 1, 2])
def test_f32_stream(n, off):
    x = synth.uniform(n, 6, 0).astype(np.float32)
    y = synth.uniform(n, 6, 1).astype(np.float32)
    xd = dev(x, off)
    yd = dev(np.zeros(n, np.float32), off)
    bs.copy(xd, yd)
    assert np.array_equal(bits(host(yd)), bits(x))
    yd = dev(y, off)
    bs.axpy(-1.3, xd, -0.25, yd)
    assert np.array_equal(bits(host(yd)), bits(oracle.axpy_f32(-1.3, x, -0.25, y)))
    d = host(bs.dot(xd, dev(y, off)))[0]
    o = oracle.dot_f32(x, y)
    scale = float(np.abs(x.astype(np.float64) * y.astype(np.float64)).sum())
    assert abs(d - o) <= 2.0 ** -40 * scale
    nr = host(bs.norm(xd))
    assert abs(nr[0] - oracle.dot_f32(x, x)) <= 2.0 ** -40 * oracle.dot_f32(x, x)


@pytest.mark.parametrize("n", SIZES)
def test_f32_cg_update(n):
    p, Ap, x, r = (synth.uniform(n, 7, s).astype(np.float32) for s in range(4))
    xd, rd = dev(x), dev(r)
    rr = host(bs.cg_update(np.float32(0.37), dev(p), dev(Ap), xd, rd))[0]
    xo, ro, rro = oracle.cg_update_f32(np.float32(0.37), p, Ap, x, r)
    assert np.array_equal(bits(host(xd)), bits(xo))
    assert np.array_equal(bits(host(rd)), bits(ro))
    assert abs(rr - rro) <= 2.0 ** -40 * rro + (0 if n else 1e-300)


def test_argument_errors():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(bs.BSError) as e:
        bs.axpy(1.0, x, 1.0, x)  # aliasing is rejected
    assert e.value.status == bs.BS_ERR_ARG


@pytest.mark.parametrize("n", [1001, 1 << 20])
def test_norm_values_outside_the_float_pair_window(n):
    """The FP64 norm squares elements with 2^-30 <= |x| < 2^31 as float pairs and
    everything else (zeros, subnormals, tiny and huge values) with DFMA."""
    x = synth.uniform(n, 9)
    sel = synth.uniform(n, 9, 1, 0.0, 1.0)
    x = np.where(sel < 0.1, x * 1e-12, x)
    x = np.where((sel >= 0.1) & (sel < 0.2), x * 1e12, x)
    x = np.where((sel >= 0.2) & (sel < 0.25), 0.0, x)
    x = np.where((sel >= 0.25) & (sel < 0.27), 5e-320, x)
    x = np.where((sel >= 0.27) & (sel < 0.3), x * 2.0 ** 31, x)
    x = np.where((sel >= 0.3) & (sel < 0.33), x * 2.0 ** -30, x)
    nr = host(bs.norm(dev(x)))
    s, sq = oracle.norm(x)
    assert rel(nr[0], s) <= 1e-13 and rel(nr[1], sq) <= 1e-13
    # small magnitudes only: the result must not be lost to the large terms
    y = synth.uniform(n, 10) * 2.0 ** -29
    nr = host(bs.norm(dev(y)))
    assert rel(nr[0], oracle.norm(y)[0]) <= 1e-13
