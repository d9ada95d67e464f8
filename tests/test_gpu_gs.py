"""GPU parity of BS6 (gather) and BS7 (scatter) and of the index maps.

Bitwise against the oracle: the CSR of Z^T (rowStarts, colIds), scatter
(including masked entries left untouched) and gather (serial sums in
ascending local order on both sides).  Meshes: structured K^3 hex meshes of
degree N with seeded element permutations -- the paper's BS6/BS7 workload
(Sec. 6.2) -- from tiny to several thousand elements, plus masked maps.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth

pytestmark = pytest.mark.gpu

MESHES = [(1, 1), (2, 1), (3, 2), (8, 3), (5, 7), (2, 15), (12, 4)]


def masked(m, frac, seed):
    ids = m.ids.copy()
    if frac > 0:
        ids[synth.uniform(ids.size, seed, 0, 0.0, 1.0) < frac] = -1
    return ids


def bits(a):
    return np.ascontiguousarray(a).view(np.uint64 if a.dtype == np.float64 else np.uint32)


@pytest.mark.parametrize("K,N", MESHES)
@pytest.mark.parametrize("frac", [0.0, 0.07])
def test_map_scatter_gather(K, N, frac):
    m = synth.Mesh(K, N, seed=K * 31 + N)
    ids = masked(m, frac, 5)
    Z = bs.Map(m.E, N, m.NG, ids)
    rs, ci = Z.export()
    ors, oci = oracle.csr(ids, m.NG)
    assert np.array_equal(rs, ors) and np.array_equal(ci, oci)
    assert np.array_equal(Z.valence().cpu().numpy(), oracle.valence(ids, m.NG))

    qG = synth.uniform(m.NG, 8)
    init = np.full(m.NL, -3.5)
    qL = torch.from_numpy(init).cuda()
    Z.scatter(torch.from_numpy(qG).cuda(), qL)
    assert np.array_equal(bits(qL.cpu().numpy()), bits(oracle.scatter(ids, qG, init)))

    ql = synth.uniform(m.NL, 9)
    g = Z.gather(torch.from_numpy(ql).cuda()).cpu().numpy()
    assert np.array_equal(bits(g), bits(oracle.gather(ids, ql, m.NG)))

    # FP32 twins
    qGf = qG.astype(np.float32)
    qLf = torch.from_numpy(init.astype(np.float32)).cuda()
    Z.scatter(torch.from_numpy(qGf).cuda(), qLf)
    assert np.array_equal(bits(qLf.cpu().numpy()),
                          bits(oracle.scatter_f32(ids, qGf, init.astype(np.float32))))
    qlf = ql.astype(np.float32)
    gf = Z.gather(torch.from_numpy(qlf).cuda()).cpu().numpy()
    assert np.array_equal(bits(gf), bits(oracle.gather_f32(ids, qlf, m.NG)))


def test_gather_of_scatter_of_ones_is_valence():
    m = synth.Mesh(6, 5, seed=3)
    Z = bs.Map(m.E, m.N, m.NG, m.ids)
    ones = torch.ones(m.NG, dtype=torch.float64, device="cuda")
    v = Z.gather(Z.scatter(ones))
    assert torch.equal(v, Z.valence().to(torch.float64))
    assert int(Z.valence().sum()) == m.NL


def test_unaligned_outputs():
    m = synth.Mesh(3, 3, seed=2)
    Z = bs.Map(m.E, m.N, m.NG, m.ids)
    qG = synth.uniform(m.NG, 1)
    buf = torch.full((m.NL + 1,), 2.0, dtype=torch.float64, device="cuda")
    Z.scatter(torch.from_numpy(qG).cuda(), buf[1:])
    assert np.array_equal(buf[1:].cpu().numpy(), oracle.scatter(m.ids, qG, np.full(m.NL, 2.0)))


def test_bad_map_rejected():
    m = synth.Mesh(2, 2, seed=1)
    ids = m.ids.copy()
    ids[5] = m.NG  # out of range
    with pytest.raises(bs.BSError) as e:
        bs.Map(m.E, m.N, m.NG, ids)
    assert e.value.status == bs.BS_ERR_ARG


@pytest.mark.parametrize("K,rows", [(3, [(0, 2500), (3000, 3100)]),
                                    (4, [(0, 1500), (2000, 2900), (5000, 5030)])])
def test_gather_row_longer_than_a_tile(K, rows):
    """A global node with more local copies than a gather tile holds (2048
    entries for the staged tiles, 1024 for the pipelined ones) is summed
    straight from the CSR; the sum order stays ascending.  Rows of 2500 and
    1500 copies (longer than one or both kinds of tile) and of 900, 100 and 30
    (long but fitting)."""
    m = synth.Mesh(K, 4, seed=1)
    ids = m.ids.copy()
    for g, (a, b) in enumerate(rows):
        ids[a:b] = 7 * g
    Z = bs.Map(m.E, m.N, m.NG, ids)
    ql = synth.uniform(m.NL, 4)
    want = oracle.gather(ids, ql, m.NG)
    g = Z.gather(torch.from_numpy(ql).cuda()).cpu().numpy()
    assert np.array_equal(bits(g), bits(want))
    gf = Z.gather(torch.from_numpy(ql.astype(np.float32)).cuda()).cpu().numpy()
    assert np.array_equal(bits(gf), bits(oracle.gather_f32(ids, ql.astype(np.float32), m.NG)))
    rs, ci = Z.export()
    ors, oci = oracle.csr(ids, m.NG)
    assert np.array_equal(rs, ors) and np.array_equal(ci, oci)


def test_gather_negative_zero_sums():
    """Sums start from +0.0: a single -0.0 copy gathers to +0.0, as in the
    definition; -0.0 + -0.0 from +0.0 is +0.0 too."""
    m = synth.Mesh(2, 2, seed=1)
    Z = bs.Map(m.E, m.N, m.NG, m.ids)
    ql = np.full(m.NL, -0.0)
    g = Z.gather(torch.from_numpy(ql).cuda()).cpu().numpy()
    assert np.array_equal(bits(g), bits(oracle.gather(m.ids, ql, m.NG)))
    assert np.all(bits(g) == 0)


@pytest.mark.parametrize("K,N", [(4, 3), (3, 2), (5, 7), (5, 4)])
def test_gather_paths_agree(K, N):
    """The gather runs the pipelined kernel (chunks of two q_L values staged by
    cp.async: 16 bytes in FP64, 8 in FP32) when q_L is aligned to a chunk --
    with N_L odd, the row holding the last local node summed from the CSR --
    and the staged-tile kernel otherwise (a q_L that starts one value into a
    buffer); every path, in both precisions, is bitwise the oracle's
    ascending-order sum, with and without masked entries (which may mask the
    last local node)."""
    m = synth.Mesh(K, N, seed=K * 7 + N)
    last_masked = m.ids.copy()
    last_masked[-1] = -1
    for ids in (m.ids, masked(m, 0.05, 11), last_masked):
        Z = bs.Map(m.E, N, m.NG, ids)
        ql = synth.uniform(m.NL, 12)
        want = oracle.gather(ids, ql, m.NG)
        buf = torch.zeros(m.NL + 1, dtype=torch.float64, device="cuda")
        buf[1:] = torch.from_numpy(ql).cuda()
        for qlt in (torch.from_numpy(ql).cuda(), buf[1:]):
            g = Z.gather(qlt).cpu().numpy()
            assert np.array_equal(bits(g), bits(want))
        qf = ql.astype(np.float32)
        want_f = oracle.gather_f32(ids, qf, m.NG)
        buf_f = torch.zeros(m.NL + 1, dtype=torch.float32, device="cuda")
        buf_f[1:] = torch.from_numpy(qf).cuda()
        for qlt in (torch.from_numpy(qf).cuda(), buf_f[1:]):
            g = Z.gather(qlt).cpu().numpy()
            assert np.array_equal(bits(g), bits(want_f))
