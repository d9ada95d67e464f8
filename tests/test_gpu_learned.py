"""GPU parity of the learned element preconditioner against the FP64 oracle.

Network (BF16 tensor cores, FP32 accumulation): the oracle runs in its bf16
mode, rounding x, the weights and the hidden activations where the GPU does,
so the two differ by FP32 accumulation order (about 1e-6 relative) plus
occasional one-ulp bf16 flips of a hidden value; outputs are compared
norm-wise at 2e-3.  Gradients: the GPU also rounds dY and relu'(.)dH to bf16
for its backward GEMMs (relative 2^-9 per entry, averaging over the batch),
so gradient tensors agree norm-wise within 1e-2 and the loss within 1e-4.
BF16x3 mode (hi + lo operands) agrees with the oracle's BF16x3 mode to FP32
accumulation order (1e-5).  Training pairs: the element-interior error from
the GPU's per-element CG against the oracle's dense Cholesky solve.
Flexible PCG: with no network, or a network whose output is zero, it is
Jacobi-PCG; with a linear correction it follows the oracle; a network trained
on the GPU needs fewer iterations than Jacobi-PCG (test_trained_network_gain);
the Jacobi judge catches a network that stalls the solve; the solve is
invariant under power-of-two scaling of b.  The tcgen05 GEMM engine gives
bitwise the results of the mma.sync one.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_10917_gb300 import bs, learned, synth
from tests import fem_ref

pytestmark = pytest.mark.gpu


def weights(D, H, seed):
    W1 = (synth.uniform(H * D, seed, 0).reshape(H, D) * np.sqrt(3.0 / D)).astype(np.float32)
    W2 = (synth.uniform(D * H, seed, 1).reshape(D, H) * np.sqrt(3.0 / H)).astype(np.float32)
    return W1, W2


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("B", [1, 37, 300])
@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("odd", [False, True])
def test_forward_matches_oracle(B, split, odd):
    D, H = 216, 256
    W1, W2 = weights(D, H, 3)
    X = synth.uniform(B * D, 4).reshape(B, D).astype(np.float32)
    net = bs.MLP(W1, W2, split=split)
    Y = net.forward(torch.from_numpy(X).cuda(), odd=odd).cpu().numpy()
    prec = oracle.PREC_BF16X3 if split else oracle.PREC_BF16
    Yo, _ = oracle.mlp_forward(W1, W2, X, prec=prec, odd=odd)
    assert rel(Y, Yo) <= (1e-5 if split else 2e-3)
    if split:  # and within its error bound of the exact network
        assert rel(Y, oracle.mlp_forward(W1, W2, X, odd=odd)[0]) <= 1e-4


@pytest.mark.parametrize("split", [False, True])
def test_gradients_match_oracle(split):
    D, H, B = 216, 256, 256
    W1, W2 = weights(D, H, 5)
    X = synth.uniform(B * D, 6).reshape(B, D).astype(np.float32)
    T = synth.uniform(B * D, 7).reshape(B, D).astype(np.float32)
    net = bs.MLP(W1, W2, split=split)
    loss, g1, g2 = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    prec = oracle.PREC_BF16X3 if split else oracle.PREC_BF16
    lo, g1o, g2o = oracle.mlp_loss_grad(W1, W2, X, T, prec=prec)
    assert abs(loss.item() - lo) <= 1e-4 * lo
    assert rel(g1.cpu().numpy(), g1o) <= 1e-2
    assert rel(g2.cpu().numpy(), g2o) <= 1e-2


@pytest.mark.parametrize("split", [False, True])
def test_small_shapes_and_padding(split):
    """D not a multiple of 32 and a narrow hidden layer."""
    D, H, B = 27, 64, 64
    W1, W2 = weights(D, H, 8)
    X = synth.uniform(B * D, 9).reshape(B, D).astype(np.float32)
    T = synth.uniform(B * D, 10).reshape(B, D).astype(np.float32)
    net = bs.MLP(W1, W2, split=split)
    prec = oracle.PREC_BF16X3 if split else oracle.PREC_BF16
    Y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    assert rel(Y, oracle.mlp_forward(W1, W2, X, prec=prec)[0]) <= 2e-3
    loss, g1, g2 = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    lo, g1o, g2o = oracle.mlp_loss_grad(W1, W2, X, T, prec=prec)
    assert rel(g1.cpu().numpy(), g1o) <= 1e-2 and rel(g2.cpu().numpy(), g2o) <= 1e-2
    w1, w2 = net.weights()
    assert np.array_equal(w1, W1) and np.array_equal(w2, W2)


def test_adam_step_matches_oracle():
    D, H, B, lr = 216, 256, 128, 1e-3
    W1, W2 = weights(D, H, 11)
    X = synth.uniform(B * D, 12).reshape(B, D).astype(np.float32)
    T = synth.uniform(B * D, 13).reshape(B, D).astype(np.float32)
    net = bs.MLP(W1, W2)
    net.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), lr)
    w1, w2 = net.weights()
    _, g1o, g2o = oracle.mlp_loss_grad(W1, W2, X, T, prec=oracle.PREC_BF16)
    z = np.zeros_like(W1)
    w1o, _, _ = oracle.adam(W1, g1o.astype(np.float32), z, z, lr, 1)
    w2o, _, _ = oracle.adam(W2, g2o.astype(np.float32), z.T.copy(), z.T.copy(), lr, 1)
    # the first Adam step moves each weight by about lr * sign(g): agreement
    # wherever the gradient is not within bf16 noise of zero
    for w, wo, go in ((w1, w1o, g1o), (w2, w2o, g2o)):
        big = np.abs(go) > 1e-2 * np.abs(go).max()
        assert np.mean(np.abs(w - wo)[big] <= 1e-2 * lr) >= 0.98
        assert np.all(np.abs(w - wo) <= 2.01 * lr)


def test_training_reduces_the_loss():
    D, H, B = 216, 256, 256
    Wt1, Wt2 = weights(D, H, 20)  # a teacher network gives the targets
    X = synth.uniform(8 * B * D, 21).reshape(8 * B, D).astype(np.float32)
    T = oracle.mlp_forward(Wt1, Wt2, X)[0].astype(np.float32)
    W1, W2 = weights(D, H, 22)
    net = bs.MLP(W1, W2)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    first = None
    for step in range(300):
        k = (step % 8) * B
        loss = net.train_step(Xd[k:k + B].contiguous(), Td[k:k + B].contiguous(), 1e-3)
        if first is None:
            first = loss.item()
    last = net.loss_grad(Xd[:B].contiguous(), Td[:B].contiguous())[0].item()
    assert last < 0.2 * first


def _problem(K, N, lam, coef=None, seed=1):
    m = synth.Mesh(K, N, seed=seed)
    Z = bs.Map(m.E, N, m.NG, m.ids)
    return m, Z, bs.Problem(Z, m.h, lam, coef)


def test_fpcg_without_network_is_jacobi_pcg():
    coef = synth.lognormal(4 ** 3, 2)
    m, Z, P = _problem(4, 3, 1e-2, coef)
    b = torch.from_numpy(synth.uniform(m.NG, 3)).cuda()
    x, info = bs.fpcg_learned(P, None, b, tol=1e-9)
    xj, ij = P.cg(b, tol=1e-9, flags=bs.BS_CG_JACOBI)
    assert abs(info["iterations"] - ij["iterations"]) <= 2
    assert torch.linalg.norm(x - xj) <= 1e-6 * torch.linalg.norm(xj)
    xo, ito, _, _ = oracle.fpcg(m.E, 3, m.h, 1e-2, m.ids, m.NG, b.cpu().numpy(), tol=1e-9,
                                coef=coef)
    assert abs(info["iterations"] - ito) <= 2


def test_fpcg_zero_network_equals_no_network():
    m, Z, P = _problem(3, 5, 1e-2)
    W1, _ = weights(216, 256, 4)
    net = bs.MLP(W1, np.zeros((216, 256), np.float32))
    b = torch.from_numpy(synth.uniform(m.NG, 5)).cuda()
    x1, i1 = bs.fpcg_learned(P, net, b, tol=1e-9)
    x2, i2 = bs.fpcg_learned(P, None, b, tol=1e-9, flags=bs.BS_CG_GRAPH)
    # z is the same; only the dot products are summed in another order
    assert abs(i1["iterations"] - i2["iterations"]) <= 1
    assert torch.linalg.norm(x1 - x2) <= 1e-8 * torch.linalg.norm(x2)


def test_fpcg_with_a_linear_correction_matches_oracle():
    """The exact element-interior map u_I -> A_II^-1 D_I u_I - u_I as the
    network's odd part (W1 = I, W2 = 2 M): the GPU's flexible PCG (BF16x3)
    follows the oracle's, meets the tolerance on the FP64 true residual and
    needs fewer iterations than Jacobi-PCG."""
    N, lam = 5, 1e-2
    coef = synth.lognormal(4 ** 3, 2)
    m, Z, P = _problem(4, N, lam, coef)
    S, M = fem_ref.element_matrices(N, m.h)  # c = 1: the map hardly depends on c
    Ae = S + lam * M
    Np = m.Np
    I = np.array([i + 6 * (j + 6 * k) for k in range(1, 5) for j in range(1, 5)
                  for i in range(1, 5)])
    Mint = np.zeros((Np, Np))
    Mint[np.ix_(I, I)] = np.linalg.solve(Ae[np.ix_(I, I)], np.diag(np.diag(Ae)[I])) - np.eye(64)
    H = 224
    W1 = np.zeros((H, Np), np.float32)
    W1[:Np] = np.eye(Np)
    W2 = np.zeros((Np, H), np.float32)
    W2[:, :Np] = 2 * Mint
    net = bs.MLP(W1, W2, split=True)
    bh = synth.uniform(m.NG, 5)
    b = torch.from_numpy(bh).cuda()
    x, info = bs.fpcg_learned(P, net, b, tol=1e-8, flags=bs.BS_FPCG_ODD)
    assert info["rc"] == 0 and info["outer"] == 0
    r = bh - oracle.apply_A(m.E, N, m.h, lam, m.ids, m.NG, x.cpu().numpy(), coef=coef)
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(bh)
    _, ito, _, _ = oracle.fpcg(m.E, N, m.h, lam, m.ids, m.NG, bh, W1, W2,
                               prec=oracle.PREC_BF16X3, odd=True, tol=1e-8, coef=coef)
    assert abs(info["iterations"] - ito) <= max(3, 0.1 * ito)
    _, ij = P.cg(b, tol=1e-8, flags=bs.BS_CG_JACOBI)
    assert info["iterations"] < 0.8 * ij["iterations"]  # 254 vs 371 in the oracle
    # the full network of this W1, W2 is the same map plus an even part: it
    # runs through the two-layer path and still converges
    _, inf2 = bs.fpcg_learned(P, net, b, tol=1e-8, maxit=20000, check=False)
    assert inf2["rc"] == 0


@pytest.mark.parametrize("N", [2, 3, 5])
def test_interior_pairs_match_oracle(N):
    K = 3
    coef = synth.lognormal(K ** 3, 2)
    m, Z, P = _problem(K, N, 1e-2, coef)
    r = synth.uniform(m.NG, 1)
    elems = np.array([0, 5, K ** 3 - 1, 13, 13], np.int32)
    X, T = bs.mlp_pairs(P, torch.from_numpy(r).cuda(), torch.from_numpy(elems).cuda(),
                        negate_odd=True)
    Xo, To = oracle.interior_pairs(m.E, N, m.h, 1e-2, m.ids, m.NG, r, elems, negate_odd=True,
                                   coef=coef)
    np.testing.assert_allclose(X.cpu().numpy(), Xo, rtol=1e-6, atol=1e-7)
    Tg = T.cpu().numpy()
    # T is an O(1) quantity (rows of X have unit mean square); at N = 2 it
    # vanishes up to rounding, so the floor is set by X's scale
    np.testing.assert_allclose(Tg, To, rtol=1e-5, atol=1e-6 * np.abs(Xo).max())
    assert np.array_equal(Tg[4], -Tg[3])  # negate_odd on a repeated element


def test_judge_switches_a_bad_network_to_jacobi():
    """A random, nonlinear correction of full size stalls flexible CG; the
    Jacobi judge restarts the solve and it still converges."""
    coef = synth.lognormal(4 ** 3, 2)
    m, Z, P = _problem(4, 3, 1e-2, coef)
    W1, W2 = weights(64, 64, 9)
    net = bs.MLP(W1, 3 * W2)
    b = torch.from_numpy(synth.uniform(m.NG, 3)).cuda()
    x, info = bs.fpcg_learned(P, net, b, tol=1e-8, maxit=20000, flags=bs.BS_CG_GRAPH)
    assert info["rc"] == 0 and info["outer"] > 0
    r = b.cpu().numpy() - oracle.apply_A(m.E, 3, m.h, 1e-2, m.ids, m.NG, x.cpu().numpy(),
                                         coef=coef)
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(b.cpu().numpy())


def test_judge_switches_near_where_the_oracle_judge_does():
    """The oracle's flexible PCG carries the same judge (checked every 8
    iterations, patience max(1024, 16 N_G^(1/3))).  On the stalling network
    both switch to Jacobi and converge.  The bf16 network's products round in
    different FP32 orders on the two sides, and a stalled flexible CG
    amplifies such differences, so the r.r histories -- and with them the
    last progress mark -- need not coincide: the switch iterations must
    agree within a tenth (at least 64 iterations), the totals within a
    quarter."""
    coef = synth.lognormal(4 ** 3, 2)
    m, Z, P = _problem(4, 3, 1e-2, coef)
    W1, W2 = weights(64, 64, 9)
    net = bs.MLP(W1, 3 * W2)
    b = synth.uniform(m.NG, 3)
    x, info = bs.fpcg_learned(P, net, torch.from_numpy(b).cuda(), tol=1e-8, maxit=20000,
                              flags=bs.BS_CG_GRAPH)
    xo, ito, hr, fb, sw = oracle.fpcg_judged(m.E, 3, m.h, 1e-2, m.ids, m.NG, b, W1, 3 * W2,
                                             prec=oracle.PREC_BF16, tol=1e-8, maxit=20000,
                                             coef=coef)
    assert info["rc"] == 0 and info["outer"] > 0 and sw > 0
    assert info["outer"] % 8 == 0
    assert abs(info["outer"] - sw) <= max(64, 0.1 * sw), (info["outer"], sw)
    assert abs(info["iterations"] - ito) <= 0.25 * ito, (info["iterations"], ito)


def test_trained_network_gain():
    """What the trained network gains over the method without it: on a
    degree-5 mesh with lognormal coefficients (lambda = 1e-2), flexible PCG
    with the trained network's odd part needs fewer iterations than
    Jacobi-PCG on a right-hand side it was not trained on."""
    N, lam = 5, 1e-2
    K = 6
    coef = synth.lognormal(K ** 3, 21)
    m, Z, P = _problem(K, N, lam, coef, seed=4)
    net, meta = learned.build_preconditioner(P, m.E, m.NG, npairs=20000, steps=40000)
    assert meta["fit_rel_error"] <= 1e-3
    b = torch.from_numpy(synth.uniform(m.NG, 4242)).cuda()
    _, ij = P.cg(b, tol=1e-8, maxit=100000, flags=bs.BS_CG_JACOBI | bs.BS_CG_GRAPH)
    x, il = bs.fpcg_learned(P, net, b, tol=1e-8, maxit=100000,
                            flags=bs.BS_FPCG_ODD | bs.BS_CG_GRAPH)
    assert il["rc"] == 0 and il["outer"] == 0
    r = b.cpu().numpy() - oracle.apply_A(m.E, N, m.h, lam, m.ids, m.NG, x.cpu().numpy(),
                                         coef=coef)
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(b.cpu().numpy())
    assert il["iterations"] <= 0.8 * ij["iterations"], (il["iterations"], ij["iterations"])


def test_fpcg_is_scale_invariant():
    """The float-pair dot products fall back to FP64 outside [2^-60, 2^60):
    a right-hand side scaled by 2^-110 (or 2^100) takes the same steps and
    gives the same solution, scaled."""
    coef = synth.lognormal(3 ** 3, 2)
    m, Z, P = _problem(3, 3, 1e-2, coef)
    W1, W2 = weights(64, 64, 4)
    net = bs.MLP(W1, (0.05 * W2).astype(np.float32), split=True)
    b = torch.from_numpy(synth.uniform(m.NG, 3)).cuda()
    x1, i1 = bs.fpcg_learned(P, net, b, tol=1e-9, flags=bs.BS_FPCG_ODD)
    for sc in (2.0 ** -110, 2.0 ** 100):
        xs, is_ = bs.fpcg_learned(P, net, b * sc, tol=1e-9, flags=bs.BS_FPCG_ODD)
        assert is_["rc"] == 0
        assert abs(is_["iterations"] - i1["iterations"]) <= 2
        # the network's input is scale-free (rms normalisation), so only
        # rounding separates the two solves
        assert torch.linalg.norm(xs / sc - x1) <= 1e-7 * torch.linalg.norm(x1)


@pytest.mark.parametrize("split", [False, True])
def test_tcgen05_engine_matches_mma_sync(split):
    """The tcgen05 GEMMs (bs_gemm_engine(1)) against the mma.sync ones: the
    forward pass of every epilogue they serve, the loss gradients and a few
    flexible-PCG iterations agree bitwise (both sum 16-wide K blocks in FP32
    in the same order); sizes with a partial 64-wide K chunk and M tails."""
    D, H = 216, 256
    W1, W2 = weights(D, H, 13)
    net = bs.MLP(W1, W2, split=split)
    X = torch.from_numpy(synth.uniform(300 * D, 14).reshape(300, D).astype(np.float32)).cuda()
    T = torch.from_numpy(synth.uniform(256 * D, 15).reshape(256, D).astype(np.float32)).cuda()
    coef = synth.lognormal(3 ** 3, 2)
    m, Z, P = _problem(3, 5, 1e-2, coef)
    b = torch.from_numpy(synth.uniform(m.NG, 16)).cuda()
    out = {}
    prev = bs.gemm_engine(-1)
    try:
        for eng in (0, 1):
            bs.gemm_engine(eng)
            y = net.forward(X)
            yo = net.forward(X, odd=True)
            loss, g1, g2 = net.loss_grad(X[:256].contiguous(), T)
            x, info = bs.fpcg_learned(P, net, b, maxit=12, flags=bs.BS_FPCG_ODD, check=False)
            x2, info2 = bs.fpcg_learned(P, net, b, maxit=12, check=False)
            out[eng] = (y, yo, loss, g1, g2, x, info["rr"], x2, info2["rr"])
    finally:
        bs.gemm_engine(prev)
    for a, c in zip(out[0], out[1]):
        if torch.is_tensor(a):
            assert torch.equal(a, c)
        else:
            assert a == c


def test_checkpoint_resumes_training_bitwise(tmp_path):
    """Training state saved after 12 Adam steps and loaded into a network
    created with other weights: 12 more steps on both give bitwise the same
    masters as 24 uninterrupted steps (weights, both Adam moments and the
    step count's bias correction all travel in the image)."""
    D, H, B = 216, 256, 128
    W1, W2 = weights(D, H, 31)
    X = torch.from_numpy(synth.uniform(24 * B * D, 32).reshape(24 * B, D).astype(np.float32)).cuda()
    T = torch.from_numpy(synth.uniform(24 * B * D, 33).reshape(24 * B, D).astype(np.float32)).cuda()
    for split in (False, True):
        a = bs.MLP(W1, W2, split=split)
        for k in range(12):
            a.train_step(X[k * B:(k + 1) * B], T[k * B:(k + 1) * B], 1e-3)
        path = tmp_path / f"state_{int(split)}.bin"
        a.save(path)
        V1, V2 = weights(D, H, 34)
        c = bs.MLP(V1, V2, split=split)
        c.load(path)
        assert all(np.array_equal(u, v) for u, v in zip(c.weights(), a.weights()))
        for k in range(12, 24):
            a.train_step(X[k * B:(k + 1) * B], T[k * B:(k + 1) * B], 1e-3)
            c.train_step(X[k * B:(k + 1) * B], T[k * B:(k + 1) * B], 1e-3)
        for u, v in zip(a.weights(), c.weights()):
            assert np.array_equal(u.view(np.uint32), v.view(np.uint32))
        ya = a.forward(X[:B]).cpu().numpy()
        yc = c.forward(X[:B]).cpu().numpy()
        assert np.array_equal(ya.view(np.uint32), yc.view(np.uint32))
    # an image of another shape or mode is refused
    img = bs.MLP(W1, W2).save_state()
    with pytest.raises(bs.BSError):
        bs.MLP(W1, W2, split=True).load_state(img)
    Wa, Wb = weights(D, 128, 35)
    with pytest.raises(bs.BSError):
        bs.MLP(Wa, Wb).load_state(img)
    with pytest.raises(bs.BSError):
        bs.MLP(W1, W2).load_state(img[:100])
