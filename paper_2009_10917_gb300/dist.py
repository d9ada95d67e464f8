"""BS6/BS7 and CG with the elements split over several ranks.

Sec. 3 sets the multi-rank gather/scatter aside as the non-trivial parallel
implementation of the method; this module is this library's form of it.

Partition.  Rank r owns a contiguous range [lo_r, hi_r) of the element
storage order (``partition``); its local vector is that slice of the
element-major q_L.  Element slabs are contiguous ranges when the storage order
runs slab by slab; any other order works too, with more shared nodes.  The
rank's map sends its elements onto the global nodes they touch, renumbered
rank-locally: the nodes the rank OWNS first (a node's owner is the highest
rank holding a copy of it), then the others, each group in ascending global
index.

Gather (BS6).  The single-domain gather sums a node's copies serially in
ascending local index, and every local index of a lower rank precedes those
of a higher one.  So a node held by ranks r_1 < r_2 < ... < r_k is summed as
a chain: r_1's ordinary gather starts it from +0, each r_i continues the
serial sum from the partial r_(i-1) sent it (``bs_gather_rows`` with a start
value), and r_k, the owner, holds bitwise the single-domain value and sends it
back to r_1 .. r_(k-1).  The exchange runs in rounds: round t passes the
partials of chain position t-1 to position t; a last round broadcasts the
owners' values.  Element slabs at least two elements thick give chains of
length two: one forward and one backward message per neighbour.

Scatter (BS7) is local: every rank holds the value of each of its nodes.

Reductions (dot, norm, r.r).  Each rank sums its owned nodes; the partials are
all-gathered and added in rank order, so every rank has the same bits (not
the single-domain bits: the order differs, within the reductions' 1e-13).

CG (Algorithm 1) strings these together with the element operator on each
rank's elements; every holder of a node updates it identically, so the
copies never drift apart.

The device steps are the library's (``bs.Map``, ``bs.Rows``, ``bs.Problem``)
through ``GpuOps``; the messages go through ``TorchComm``
(``torch.distributed``: NCCL for device buffers, gloo for host ones), or
through ``run_lockstep``, which advances every rank of one process round by
round (several ranks on one GPU, with no kernel waiting on another).
"""
from __future__ import annotations

import numpy as np


def partition(E: int, nranks: int):
    """Balanced contiguous ranges of the element storage order."""
    b = [E * r // nranks for r in range(nranks + 1)]
    return [(b[r], b[r + 1]) for r in range(nranks)]


def touched_nodes(l2g_part: np.ndarray) -> np.ndarray:
    """Sorted global indices of the nodes a rank's elements touch."""
    ids = np.asarray(l2g_part)
    return np.unique(ids[ids >= 0]).astype(np.int64)


class Round:
    """One forward round: partials sent on (my chain position t - 1) and
    received (my position t), local rows per peer in ascending global index;
    ``cont`` is the receive rows of all peers, peers ascending (the order of
    the start values)."""

    def __init__(self, send, recv):
        self.send, self.recv = send, recv
        self.cont = (np.concatenate([recv[q] for q in sorted(recv)]).astype(np.int32)
                     if recv else np.zeros(0, np.int32))


class Plan:
    """The exchange plan of one rank, from its slice of the local-to-global
    map and the touched-node lists of all ranks (rank order).

    Attributes: rank, nranks, nodes (global index of each rank-local node;
    owned first), n_owned, ids (the rank-local map, -1 stays masked), depth
    (longest chain of holders over the whole mesh), rounds (depth - 1 forward
    rounds), final_send / final_recv (owner broadcast, local rows per peer).
    """

    def __init__(self, rank: int, l2g_part: np.ndarray, touched_all):
        P = len(touched_all)
        self.rank, self.nranks = int(rank), P
        mine = np.asarray(touched_all[rank], dtype=np.int64)
        n = mine.size
        held = np.zeros((n, P), dtype=bool)
        for q, tq in enumerate(touched_all):
            tq = np.asarray(tq, dtype=np.int64)
            if tq.size == 0 or n == 0:
                continue
            i = np.minimum(np.searchsorted(tq, mine), tq.size - 1)
            held[:, q] = tq[i] == mine
        allnodes = np.concatenate([np.asarray(t, dtype=np.int64) for t in touched_all])
        self.depth = int(np.unique(allnodes, return_counts=True)[1].max()) if allnodes.size else 1
        pos = held[:, :rank].sum(axis=1)                 # my place in each node's chain
        owner = P - 1 - np.argmax(held[:, ::-1], axis=1)  # highest holder
        prev = np.full(n, -1, np.int64)
        for q in range(rank):
            prev = np.where(held[:, q], q, prev)
        nxt = np.full(n, -1, np.int64)
        for q in range(P - 1, rank, -1):
            nxt = np.where(held[:, q], q, nxt)
        owned = owner == rank
        order = np.concatenate([np.flatnonzero(owned), np.flatnonzero(~owned)])
        loc = np.empty(n, np.int64)
        loc[order] = np.arange(n)
        self.nodes, self.n_owned = mine[order], int(owned.sum())
        ids = np.asarray(l2g_part)
        self.ids = np.full(ids.size, -1, np.int32)
        m = ids >= 0
        self.ids[m] = loc[np.searchsorted(mine, ids[m])]

        def rows(sel):  # local rows of the selected nodes, ascending global index
            return loc[np.flatnonzero(sel)].astype(np.int32)

        self.rounds = []
        for t in range(1, self.depth):
            send = {int(q): rows((pos == t - 1) & (nxt == q)) for q in range(rank + 1, P)}
            recv = {int(q): rows((pos == t) & (prev == q)) for q in range(rank)}
            self.rounds.append(Round({q: r for q, r in send.items() if r.size},
                                     {q: r for q, r in recv.items() if r.size}))
        self.final_send = {int(q): rows(owned & held[:, q]) for q in range(P) if q != rank}
        self.final_send = {q: r for q, r in self.final_send.items() if r.size}
        self.final_recv = {int(q): rows(owner == q) for q in range(P) if q != rank}
        self.final_recv = {q: r for q, r in self.final_recv.items() if r.size}

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.size)

    def recv_sizes(self):
        """Message sizes this rank receives, per exchange (rounds, then the
        owner broadcast)."""
        out = [{q: int(r.size) for q, r in rd.recv.items()} for rd in self.rounds]
        out.append({q: int(r.size) for q, r in self.final_recv.items()})
        return out


def make_plan(rank: int, l2g_part: np.ndarray, comm) -> Plan:
    """Plan of this rank; comm.allgather_array shares the touched-node lists."""
    return Plan(rank, l2g_part, comm.allgather_array(touched_nodes(l2g_part)))


class Part:
    """One rank's device objects for a plan: its map, the row sets of every
    exchange, and (for CG) its element operator."""

    def __init__(self, plan: Plan, ops, E_r: int, N: int, coef=None):
        self.plan, self.ops, self.E, self.N = plan, ops, int(E_r), int(N)
        self.coef = None if coef is None else np.ascontiguousarray(coef, dtype=np.float64)
        self.problem = None
        self.map = ops.map(E_r, N, plan.n_nodes, plan.ids)
        self.send_rows = [{q: ops.rows(self.map, r) for q, r in rd.send.items()}
                          for rd in plan.rounds]
        self.cont_rows = [ops.rows(self.map, rd.cont) for rd in plan.rounds]
        self.final_send = {q: ops.rows(self.map, r) for q, r in plan.final_send.items()}
        self.final_recv = {q: ops.rows(self.map, r) for q, r in plan.final_recv.items()}


def gather_steps(part: Part, qL, qG):
    """The multi-rank gather of one rank as a generator of requests: it
    yields ("msg", {peer: buffer}) for each exchange and is sent the buffers
    it receives ({peer: buffer}); qG (the rank's nodes) holds the result when
    it finishes."""
    ops, plan = part.ops, part.plan
    ops.gather(part.map, qL, qG)  # from +0: right wherever this rank comes first
    for t, rd in enumerate(plan.rounds):
        recv = yield ("msg", {q: ops.pack(h, qG) for q, h in part.send_rows[t].items()})
        if rd.recv:
            start = ops.concat([recv[q] for q in sorted(rd.recv)])
            ops.gather_rows(part.cont_rows[t], qL, start, qG)
    recv = yield ("msg", {q: ops.pack(h, qG) for q, h in part.final_send.items()})
    for q in sorted(part.final_recv):
        ops.unpack(part.final_recv[q], recv[q], qG)


def allsum(values) -> float:
    """Rank-ordered sum of the per-rank partials (the same bits everywhere)."""
    s = 0.0
    for v in values:
        s = s + float(v)
    return s


def reduce_steps(value):
    """A scalar all-reduce as a generator request: yields ("sum", value) and
    returns the rank-ordered sum over all ranks."""
    total = yield ("sum", float(value))
    return total


def run_steps(gen, comm, plan: Plan):
    """Drive one rank's generator over a communicator: exchanges through
    comm.exchange (sizes from the plan, one gather after another), scalar
    sums through comm.allgather_float.  Returns the generator's value."""
    sizes = plan.recv_sizes()
    k = 0
    try:
        req = next(gen)
        while True:
            kind, payload = req
            if kind == "sum":
                reply = allsum(comm.allgather_float(payload))
            else:
                reply = comm.exchange(payload, sizes[k % len(sizes)])
                k += 1
            req = gen.send(reply)
    except StopIteration as stop:
        return stop.value


def run_lockstep(gens, plans):
    """Drive the generators of all ranks of one process together: each step
    collects every rank's request (all of one kind), routes the messages or
    forms the sum, and resumes every rank.  Returns the generators' values."""
    P = len(gens)
    sizes = [p.recv_sizes() for p in plans]
    out = [None] * P
    reqs = []
    for r, g in enumerate(gens):
        try:
            reqs.append(next(g))
        except StopIteration as stop:
            out[r] = stop.value
            reqs.append(None)
    k = 0
    while any(q is not None for q in reqs):
        if any(q is None for q in reqs) or len({q[0] for q in reqs}) != 1:
            raise RuntimeError("ranks out of step")
        if reqs[0][0] == "sum":
            total = allsum(q[1] for q in reqs)
            replies = [total] * P
        else:
            replies = [{} for _ in range(P)]
            for src in range(P):
                for dst, buf in reqs[src][1].items():
                    replies[dst][src] = buf
            for r in range(P):
                want = sizes[r][k % len(sizes[r])]
                got = {q: len(b) for q, b in replies[r].items()}
                if got != want:
                    raise RuntimeError(f"rank {r}: messages {got} do not match the plan {want}")
            k += 1
        for r, g in enumerate(gens):
            try:
                reqs[r] = g.send(replies[r])
            except StopIteration as stop:
                out[r] = stop.value
                reqs[r] = None
    return out


def gather(part: Part, qL, qG, comm):
    """BS6 over the ranks of `comm` (every rank calls it)."""
    run_steps(gather_steps(part, qL, qG), comm, part.plan)
    return qG


def dot_steps(part: Part, x, y):
    """x.y over the ranks (owned nodes, rank-ordered sum) as a generator."""
    v = yield from reduce_steps(part.ops.dot_prefix(x, y, part.plan.n_owned))
    return v


def cg_steps(part: Part, b, x, tol: float, maxit: int, hist=None):
    """Algorithm 1 on one rank as a generator of requests (gather exchanges
    and scalar sums).  b, x: this rank's nodes (x is overwritten, the solve
    starts from 0).  The value is (iterations, r.r, b.b); hist, if a list,
    receives (alpha, beta, r.r) per iteration."""
    ops = part.ops
    ops.fill(x, 0.0)
    r = ops.copy(b)
    p = ops.copy(b)
    bb = yield from dot_steps(part, b, b)
    rr = bb
    eps = tol * tol * bb
    pL = ops.local_vector(part)
    wL = ops.local_vector(part)
    Ap = ops.zeros_like(b)
    it = 0
    while it < maxit and rr > eps:
        ops.scatter(part.map, p, pL)
        ops.apply_local(part, pL, wL)
        yield from gather_steps(part, wL, Ap)
        pAp = yield from dot_steps(part, p, Ap)
        if not (pAp > 0.0) or not np.isfinite(pAp):
            raise FloatingPointError("CG breakdown: p.Ap <= 0 or not finite")
        alpha = rr / pAp
        ops.update(alpha, p, Ap, x, r)
        rr_new = yield from dot_steps(part, r, r)
        beta = rr_new / rr
        ops.axpy(1.0, r, beta, p)
        if hist is not None:
            hist.append((alpha, beta, rr_new))
        rr = rr_new
        it += 1
    return it, rr, bb


class TorchComm:
    """Messages and reductions over torch.distributed (the default process
    group): point-to-point buffers in batches, all-gathers of scalars and of
    host arrays.  device: where received buffers live (a CUDA device for
    NCCL, "cpu" for gloo)."""

    def __init__(self, device="cpu"):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.device = torch, dist, device
        self.rank, self.size = dist.get_rank(), dist.get_world_size()

    def exchange(self, sends, recv_sizes):
        torch, dist = self.torch, self.dist
        ops, recv = [], {}
        for q in sorted(recv_sizes):
            recv[q] = torch.empty(recv_sizes[q], dtype=torch.float64, device=self.device)
            ops.append(dist.P2POp(dist.irecv, recv[q], q))
        for q in sorted(sends):
            ops.append(dist.P2POp(dist.isend, sends[q].contiguous(), q))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return recv

    def allgather_float(self, v):
        t = self.torch.tensor([float(v)], dtype=self.torch.float64, device=self.device)
        out = [self.torch.empty_like(t) for _ in range(self.size)]
        self.dist.all_gather(out, t)
        return [float(o.item()) for o in out]

    def allgather_array(self, a):
        out = [None] * self.size
        self.dist.all_gather_object(out, np.asarray(a))
        return out


class GpuOps:
    """The device steps through the library (bs.Map, bs.Rows, bs.Problem)."""

    def __init__(self, h: float = 1.0, lam: float = 1.0):
        import torch

        from . import bs
        self.bs, self.torch, self.h, self.lam = bs, torch, h, lam

    def map(self, E, N, NG, ids):
        return self.bs.Map(E, N, NG, ids)

    def rows(self, m, rows):
        return self.bs.Rows(m, rows)

    def gather(self, m, qL, qG):
        m.gather(qL, qG)

    def scatter(self, m, qG, qL):
        m.scatter(qG, qL)

    def gather_rows(self, rs, qL, start, qG):
        rs.gather(qL, qG, start)

    def pack(self, rs, qG):
        return rs.pack(qG)

    def unpack(self, rs, buf, qG):
        rs.unpack(buf, qG)

    def concat(self, bufs):
        return bufs[0] if len(bufs) == 1 else self.torch.cat(bufs)

    # vectors and CG steps
    def problem(self, part):
        if part.problem is None:
            part.problem = self.bs.Problem(part.map, self.h, self.lam, part.coef)
        return part.problem

    def local_vector(self, part):
        return self.torch.empty(part.map.NL, dtype=self.torch.float64, device="cuda")

    def zeros_like(self, v):
        return self.torch.zeros_like(v)

    def copy(self, v):
        return self.bs.copy(v)

    def fill(self, v, value):
        v.fill_(value)

    def apply_local(self, part, uL, wL):
        self.problem(part).apply_local(uL, wL)

    def dot_prefix(self, x, y, n):
        return self.bs.dot(x[:n], y[:n]).item()

    def update(self, alpha, p, Ap, x, r):
        self.bs.cg_update(alpha, p, Ap, x, r)

    def axpy(self, alpha, x, beta, y):
        self.bs.axpy(alpha, x, beta, y)
