"""The multi-rank gather and CG with the library's device steps, several
ranks advanced together in one process on one GPU (dist.run_lockstep: every
rank's kernels finish before any message moves, so no kernel waits on
another).  Through the C ABI: bs_gather (first holders), bs_gather_rows (the
continued chain sums), bs_rows_pack / bs_rows_unpack (messages), bs_scatter,
bs_apply_local, bs_dot, bs_cg_update, bs_axpy.

- The gather is bitwise the oracle's single-domain gather on every rank's
  nodes (element slabs; the permuted order with long chains; masked entries;
  the benchmark's degree 7 on a 24^3 mesh cut into four slabs).
- bs_gather_rows with and without start values against the definition on
  the host; pack and unpack are bitwise index moves.
- CG over three ranks follows the oracle's Algorithm 1 within 1e-11 per
  iteration (alpha, beta, r.r) over 30 iterations, x within 1e-10.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, synth
from paper_2009_10917_gb300 import dist as D

pytestmark = pytest.mark.gpu


def _setup(K, N, permute, masked, P, seed=3, lam=1.0):
    m = synth.Mesh(K, N, seed=seed, permute=permute)
    ids = m.ids.copy()
    if masked > 0:
        ids[synth.uniform(ids.size, seed, 5, 0.0, 1.0) < masked] = -1
    parts = D.partition(m.E, P)
    slices = [ids[lo * m.Np:hi * m.Np] for lo, hi in parts]
    touched = [D.touched_nodes(s) for s in slices]
    plans = [D.Plan(r, slices[r], touched) for r in range(P)]
    ops = D.GpuOps(h=m.h, lam=lam)
    prts = [D.Part(pl, ops, hi - lo, N) for pl, (lo, hi) in zip(plans, parts)]
    return m, ids, parts, plans, prts


@pytest.mark.parametrize("K,N,permute,masked,P", [
    (4, 3, False, 0.0, 2), (6, 2, False, 0.05, 3), (4, 3, True, 0.0, 3), (3, 4, True, 0.05, 5),
    (24, 7, False, 0.0, 4)])
def test_gather_over_ranks_is_bitwise_the_single_domain_gather(K, N, permute, masked, P):
    m, ids, parts, plans, prts = _setup(K, N, permute, masked, P)
    ql = synth.uniform(m.NL, 7)
    ql[::13] = -0.0
    want = oracle.gather(ids, ql, m.NG)
    qGs = [torch.full((pl.n_nodes,), float("nan"), dtype=torch.float64, device="cuda")
           for pl in plans]
    qls = [torch.from_numpy(ql[lo * m.Np:hi * m.Np].copy()).cuda() for lo, hi in parts]
    D.run_lockstep([D.gather_steps(pt, a, q) for pt, a, q in zip(prts, qls, qGs)], plans)
    for pl, q in zip(plans, qGs):
        assert np.array_equal(q.cpu().numpy().view(np.uint64), want[pl.nodes].view(np.uint64))


def test_rows_gather_pack_unpack():
    m = synth.Mesh(3, 3, seed=5)
    Z = bs.Map(m.E, m.N, m.NG, m.ids)
    rows = synth.permutation(m.NG, 6)[: m.NG // 3].astype(np.int32)
    rs = bs.Rows(Z, rows)
    ql = synth.uniform(m.NL, 8)
    start = synth.uniform(rows.size, 9)
    qG = torch.full((m.NG,), 5.5, dtype=torch.float64, device="cuda")
    rs.gather(torch.from_numpy(ql).cuda(), qG, torch.from_numpy(start).cuda())
    want = np.full(m.NG, 5.5)
    for i, g in enumerate(rows):  # the definition, one row at a time
        s = start[i]
        for l in np.flatnonzero(m.ids == g):
            s = s + ql[l]
        want[g] = s
    assert np.array_equal(qG.cpu().numpy().view(np.uint64), want.view(np.uint64))
    rs.gather(torch.from_numpy(ql).cuda(), qG)  # from +0: the gather's values
    full = oracle.gather(m.ids, ql, m.NG)
    assert np.array_equal(qG.cpu().numpy()[rows], full[rows])
    buf = rs.pack(qG)
    assert np.array_equal(buf.cpu().numpy(), qG.cpu().numpy()[rows])
    other = torch.zeros(m.NG, dtype=torch.float64, device="cuda")
    rs.unpack(buf, other)
    o = other.cpu().numpy()
    assert np.array_equal(o[rows], full[rows]) and np.all(np.delete(o, rows) == 0.0)
    with pytest.raises(bs.BSError):
        bs.Rows(Z, np.array([1, 1], np.int32))  # a repeated row
    with pytest.raises(bs.BSError):
        bs.Rows(Z, np.array([m.NG], np.int32))  # out of range


def test_cg_over_ranks_follows_the_single_domain_cg():
    m, ids, parts, plans, prts = _setup(4, 3, True, 0.0, 3)
    b = synth.uniform(m.NG, 10, stream=7)
    xs = [torch.zeros(pl.n_nodes, dtype=torch.float64, device="cuda") for pl in plans]
    hists = [[] for _ in plans]
    gens = [D.cg_steps(pt, torch.from_numpy(b[pl.nodes].copy()).cuda(), x, 0.0, 30, h)
            for pt, pl, x, h in zip(prts, plans, xs, hists)]
    res = D.run_lockstep(gens, plans)
    xo, it, ha, hb, hr = oracle.cg(m.E, m.N, m.h, 1.0, ids, m.NG, b, tol=0.0, maxit=30,
                                   fixed_iters=True)
    for (itr, rr, bb), h, pl, x in zip(res, hists, plans, xs):
        assert itr == 30
        h = np.array(h)
        assert np.all(np.abs(h[:, 0] - ha) <= 1e-11 * np.abs(ha))
        assert np.all(np.abs(h[:, 1] - hb) <= 1e-11 * np.abs(hb))
        assert np.all(np.abs(h[:, 2] - hr[1:]) <= 1e-11 * np.abs(hr[1:]))
        xn = x.cpu().numpy()
        assert np.linalg.norm(xn - xo[pl.nodes]) <= 1e-10 * np.linalg.norm(xo[pl.nodes])
    assert hists[0] == hists[1] == hists[2]  # every rank takes the same steps
