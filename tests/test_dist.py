"""The multi-rank gather/scatter and CG (paper_2009_10917_gb300/dist.py) on
CPU ranks, against the single-domain oracle.

The device steps are the host stand-ins of tests/dist_cpu_ops.py (plain
definitions and the oracle), so what is tested here is the exchange logic:
the partition, the chains of holders, the message lists, the rounds and the
rank-ordered reductions.

- The gather over P ranks is BITWISE the oracle's single-domain gather
  (ascending local index), for element slabs (natural storage order: chains
  of two) and for the seeded permuted order (chains up to eight ranks long),
  with masked entries, and every holder of a node ends with the owner's bits.
- Inner products over owned nodes agree with the oracle's Dot2 within 1e-13.
- CG over the ranks follows the oracle's single-domain Algorithm 1: alpha,
  beta and r.r within 1e-11 relative per iteration over 30 iterations (they
  differ only by the reductions' order), x within 1e-10.
- Two and three gloo processes run the same through torch.distributed.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2009_10917_gb300 import dist as D
from paper_2009_10917_gb300 import synth
from tests.dist_cpu_ops import CpuOps


def _mesh(K, N, permute, masked=0.0, seed=3):
    m = synth.Mesh(K, N, seed=seed, permute=permute)
    ids = m.ids.copy()
    if masked > 0:
        ids[synth.uniform(ids.size, seed, 5, 0.0, 1.0) < masked] = -1
    return m, ids


def _plans(ids, E, Np, P):
    parts = D.partition(E, P)
    slices = [ids[lo * Np:hi * Np] for lo, hi in parts]
    touched = [D.touched_nodes(s) for s in slices]
    return parts, slices, [D.Plan(r, slices[r], touched) for r in range(P)]


@pytest.mark.parametrize("K,N,permute,P", [(4, 3, False, 2), (6, 2, False, 4), (4, 3, True, 3),
                                            (3, 4, True, 5)])
def test_plan_invariants(K, N, permute, P):
    m, ids = _mesh(K, N, permute)
    parts, slices, plans = _plans(ids, m.E, m.Np, P)
    owned = np.concatenate([p.nodes[:p.n_owned] for p in plans])
    touched = np.unique(ids[ids >= 0])
    assert np.array_equal(np.sort(owned), touched)  # every node has exactly one owner
    for p, s in zip(plans, slices):
        assert np.array_equal(p.nodes[p.ids[s >= 0]], s[s >= 0])  # local map is the global one
        assert np.all(np.diff(p.nodes[:p.n_owned]) > 0)
        assert np.all(np.diff(p.nodes[p.n_owned:]) > 0)
    for a in plans:  # every message list matches its receiver's, node for node
        for t, rd in enumerate(a.rounds):
            for q, rows in rd.send.items():
                assert np.array_equal(a.nodes[rows], plans[q].nodes[plans[q].rounds[t].recv[a.rank]])
        for q, rows in a.final_send.items():
            assert np.array_equal(a.nodes[rows], plans[q].nodes[plans[q].final_recv[a.rank]])
    if not permute and K // P >= 2:
        assert plans[0].depth == 2  # slabs at least two elements thick


def _lockstep_gather(m, ids, P, ql):
    parts, slices, plans = _plans(ids, m.E, m.Np, P)
    ops = CpuOps()
    prts = [D.Part(pl, ops, hi - lo, m.N) for pl, (lo, hi) in zip(plans, parts)]
    qGs = [torch.full((pl.n_nodes,), np.nan, dtype=torch.float64) for pl in plans]
    gens = [D.gather_steps(pt, torch.from_numpy(ql[lo * m.Np:hi * m.Np].copy()), q)
            for pt, (lo, hi), q in zip(prts, parts, qGs)]
    D.run_lockstep(gens, plans)
    return plans, [q.numpy() for q in qGs]


@pytest.mark.parametrize("K,N,permute,masked,P", [
    (4, 3, False, 0.0, 2), (6, 2, False, 0.05, 3), (4, 3, True, 0.0, 2), (4, 3, True, 0.05, 3),
    (3, 4, True, 0.0, 5), (5, 1, True, 0.0, 8)])
def test_lockstep_gather_is_bitwise_the_single_domain_gather(K, N, permute, masked, P):
    m, ids = _mesh(K, N, permute, masked)
    ql = synth.uniform(m.NL, 7)
    ql[::11] = -0.0  # signed zeros take the +0 start
    want = oracle.gather(ids, ql, m.NG)
    plans, qGs = _lockstep_gather(m, ids, P, ql)
    for pl, q in zip(plans, qGs):
        assert np.array_equal(q.view(np.uint64), want[pl.nodes].view(np.uint64))
    if permute and P >= 3:
        assert plans[0].depth >= 3  # long chains were exercised


def _rank_main(rank, world, port, K, N, permute, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, ids = _mesh(K, N, permute, 0.0)
        comm = D.TorchComm("cpu")
        lo, hi = D.partition(m.E, world)[rank]
        plan = D.make_plan(rank, ids[lo * m.Np:hi * m.Np], comm)
        ops = CpuOps(h=m.h, lam=1.0)
        part = D.Part(plan, ops, hi - lo, N)
        ql = synth.uniform(m.NL, 8)
        qG = torch.zeros(plan.n_nodes, dtype=torch.float64)
        D.gather(part, torch.from_numpy(ql[lo * m.Np:hi * m.Np].copy()), qG, comm)
        g_ok = np.array_equal(qG.numpy().view(np.uint64),
                              oracle.gather(ids, ql, m.NG)[plan.nodes].view(np.uint64))
        x = synth.uniform(m.NG, 9, 0)
        y = synth.uniform(m.NG, 9, 1)
        d = D.run_steps(D.dot_steps(part, torch.from_numpy(x[plan.nodes].copy()),
                                    torch.from_numpy(y[plan.nodes].copy())), comm, plan)
        b = synth.uniform(m.NG, 10, stream=7)
        xl = torch.zeros(plan.n_nodes, dtype=torch.float64)
        hist = []
        it, rr, bb = D.run_steps(D.cg_steps(part, torch.from_numpy(b[plan.nodes].copy()), xl,
                                            0.0, 30, hist), comm, plan)
        out[rank] = {"gather_bitwise": g_ok, "dot": d, "hist": hist, "it": it,
                     "nodes": plan.nodes, "x": xl.numpy().copy()}
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,K,N,permute", [(2, 4, 3, False), (3, 3, 3, True)])
def test_gloo_ranks_gather_dot_and_cg(world, K, N, permute):
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), K, N, permute, out),
                       nprocs=world, join=True, start_method="spawn")
    m, ids = _mesh(K, N, permute, 0.0)
    x = synth.uniform(m.NG, 9, 0)
    y = synth.uniform(m.NG, 9, 1)
    o = oracle.dot(x, y)
    b = synth.uniform(m.NG, 10, stream=7)
    xo, it, ha, hb, hr = oracle.cg(m.E, N, m.h, 1.0, ids, m.NG, b, tol=0.0, maxit=30,
                                   fixed_iters=True)
    for r in range(world):
        res = out[r]
        assert res["gather_bitwise"]
        assert res["dot"] == out[0]["dot"]  # the same bits on every rank
        assert abs(res["dot"] - o) <= 1e-13 * abs(o)
        assert res["it"] == 30
        h = np.array(res["hist"])
        assert np.all(np.abs(h[:, 0] - ha) <= 1e-11 * np.abs(ha))
        assert np.all(np.abs(h[:, 1] - hb) <= 1e-11 * np.abs(hb))
        assert np.all(np.abs(h[:, 2] - hr[1:]) <= 1e-11 * np.abs(hr[1:]))
        assert np.linalg.norm(res["x"] - xo[res["nodes"]]) <= 1e-10 * np.linalg.norm(xo[res["nodes"]])
