"""Host stand-ins for the device steps of the multi-rank gather and CG, so the
exchange logic of paper_2009_10917_gb300/dist.py runs on CPU ranks (gloo).

Each step is the plain definition: a gather adds a row's copies one at a
time in ascending local index (numpy's unbuffered ``add.at`` walks the index
array in order), starting from +0 or from the given start values; pack and
unpack are index moves; the element operator, the inner products and the CG
update are the oracle's.  Buffers are CPU torch tensors (what gloo sends).
"""
from types import SimpleNamespace

import numpy as np
import torch

import oracle


class CpuOps:
    def __init__(self, h: float = 1.0, lam: float = 1.0):
        self.h, self.lam = h, lam

    def map(self, E, N, NG, ids):
        ids = np.asarray(ids, dtype=np.int64)
        return SimpleNamespace(E=E, N=N, NG=NG, NL=ids.size, ids=ids)

    def rows(self, m, rows):
        return SimpleNamespace(m=m, rows=np.asarray(rows, dtype=np.int64))

    def gather(self, m, qL, qG):
        q, ql = qG.numpy(), qL.numpy()
        q[:] = 0.0
        ok = m.ids >= 0
        np.add.at(q, m.ids[ok], ql[ok])

    def scatter(self, m, qG, qL):
        ok = m.ids >= 0
        qL.numpy()[ok] = qG.numpy()[m.ids[ok]]

    def gather_rows(self, rs, qL, start, qG):
        q, ql = qG.numpy(), qL.numpy()
        q[rs.rows] = start.numpy() if start is not None else 0.0
        sel = np.isin(rs.m.ids, rs.rows)
        np.add.at(q, rs.m.ids[sel], ql[sel])

    def pack(self, rs, qG):
        return torch.from_numpy(qG.numpy()[rs.rows].copy())

    def unpack(self, rs, buf, qG):
        qG.numpy()[rs.rows] = buf.numpy()

    def concat(self, bufs):
        return torch.cat(bufs)

    def local_vector(self, part):
        return torch.zeros(part.map.NL, dtype=torch.float64)

    def zeros_like(self, v):
        return torch.zeros_like(v)

    def copy(self, v):
        return v.clone()

    def fill(self, v, value):
        v.fill_(value)

    def apply_local(self, part, uL, wL):
        wL.numpy()[:] = oracle.apply_local(part.E, part.N, self.h, self.lam, uL.numpy(),
                                           part.coef)

    def dot_prefix(self, x, y, n):
        return oracle.dot(x.numpy()[:n], y.numpy()[:n]) if n else 0.0

    def update(self, alpha, p, Ap, x, r):
        xo, ro, _ = oracle.cg_update(alpha, p.numpy(), Ap.numpy(), x.numpy(), r.numpy())
        x.numpy()[:] = xo
        r.numpy()[:] = ro

    def axpy(self, alpha, x, beta, y):
        y.numpy()[:] = oracle.axpy(alpha, x.numpy(), beta, y.numpy())
