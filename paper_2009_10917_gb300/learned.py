"""Training driver of the learned element preconditioner.

Every arithmetic step runs in libbs kernels (Jacobi-PCG, the operator, the
pair kernel, the network's forward/backward and Adam); this module only
sequences the calls and slices device tensors into batches.

Pairs: residuals r_k of the first iterations k of Jacobi-PCG solves with
random right-hand sides (the solves "generate" the data), and for a random
subset of elements the element-interior error e_I = A_II^-1 r_I
(bs_mlp_pairs).  Early residuals are close to white noise, which keeps the
regression well conditioned; the map being learned is local and linear, so
it does not depend on which residuals are shown.  Every other pair is
negated: (-r, -e) is as valid as (r, e), and the sign symmetry drives the
even part of the ReLU network towards zero.

Training: Adam on the mean squared error, batches of 256, cosine learning
rate from lr to 0 over the given steps, in BF16x3 mode so that the fitted
map keeps about 16 bits per weight.  The solver then uses the network's odd
part W2 W1 x / 2 (bs.BS_FPCG_ODD).
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import bs, synth


def jacobi_residual(problem: "bs.Problem", b: torch.Tensor, k: int) -> torch.Tensor:
    """r_k = b - A x_k after k Jacobi-PCG iterations from x_0 = 0."""
    if k == 0:
        return b.clone()
    x, _ = problem.cg(b, maxit=k, flags=bs.BS_CG_JACOBI | bs.BS_CG_FIXED_ITERS)
    Ax = problem.apply_A(x)
    bs.axpy(1.0, b, -1.0, Ax)
    return Ax


def make_pairs(problem: "bs.Problem", E: int, NG: int, npairs: int = 20000,
               ks=(0, 1, 2, 3, 5), seed: int = 0):
    """npairs training pairs (X, T) on the device, from Jacobi-PCG residuals
    at iterations ks of solves with b ~ U[-1, 1)^N_G (seeded)."""
    per = -(-npairs // len(ks))
    nb = max(1, -(-per // E))
    Xs, Ts, have = [], [], 0
    for s_ in range(nb):
        b = torch.from_numpy(synth.uniform(NG, 1000 + 97 * seed + s_, stream=5)).cuda()
        for k in ks:
            take = min(E, per - s_ * E, npairs - have)
            if take <= 0:
                continue
            r = jacobi_residual(problem, b, k)
            pick = synth.permutation(E, 2000 + 31 * s_ + k + 7919 * seed)[:take]
            elems = torch.from_numpy(pick.astype(np.int32)).cuda()
            X, T = bs.mlp_pairs(problem, r, elems, negate_odd=True)
            Xs.append(X)
            Ts.append(T)
            have += take
    return torch.cat(Xs), torch.cat(Ts)


def train(X: torch.Tensor, T: torch.Tensor, H: int = 256, steps: int = 40000,
          lr: float = 2e-3, batch: int = 256, seed: int = 0) -> "bs.MLP":
    """Train y = W2 relu(W1 x) (BF16x3) on the pairs; W1 ~ U(+-sqrt(3/D)),
    W2 = 0.  Returns the bs.MLP."""
    n, D = X.shape
    if n < batch:
        raise ValueError(f"need at least {batch} pairs, got {n}")
    order = torch.from_numpy(synth.permutation(n, 77 + seed).astype(np.int64)).to(X.device)
    m = n // batch * batch
    Xs, Ts = X[order][:m].contiguous(), T[order][:m].contiguous()
    W1 = (synth.uniform(H * D, 500 + seed, 0).reshape(H, D) * math.sqrt(3.0 / D))
    net = bs.MLP(W1.astype(np.float32), np.zeros((D, H), np.float32), split=True)
    loss = torch.zeros(1, dtype=torch.float64, device=X.device)
    nbat = m // batch
    for t in range(steps):
        k = (t % nbat) * batch
        lr_t = max(lr * 0.5 * (1.0 + math.cos(math.pi * t / steps)), 1e-9)
        net.train_step(Xs[k:k + batch], Ts[k:k + batch], lr_t, loss)
    return net


def fit_error(net: "bs.MLP", X: torch.Tensor, T: torch.Tensor, rows: int = 4096) -> float:
    """Relative error ||g(X) - T|| / ||T|| of the odd part g on the first rows."""
    Xr, Tr = X[:rows].contiguous(), T[:rows].contiguous()
    Y = net.forward(Xr, odd=True)
    return float(torch.linalg.norm(Y - Tr) / torch.linalg.norm(Tr))


def build_preconditioner(problem, E, NG, npairs=20000, steps=40000, lr=2e-3, seed=0):
    """Pairs + training; returns (net, timings and fit)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, T = make_pairs(problem, E, NG, npairs=npairs, seed=seed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = train(X, T, steps=steps, lr=lr, seed=seed)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return net, {"pairs": int(X.shape[0]), "pairs_seconds": round(t1 - t0, 3),
                 "train_steps": steps, "train_seconds": round(t2 - t1, 3),
                 "fit_rel_error": fit_error(net, X, T)}
