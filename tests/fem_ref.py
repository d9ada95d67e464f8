"""Dense numpy reference of the spectral-element operator, for pinning tests.

Built independently of the C oracle and of the GPU library: GLL nodes come
from numpy's Legendre class (roots of P_N'), Lagrange derivatives from
numpy polynomial algebra, and the element matrices from Kronecker products
(eqs. assembled_stiff / assembled_mass with collocated GLL quadrature).
Only for tiny meshes: everything is a dense matrix.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as L
from numpy.polynomial import polynomial as P


def gll_np(N: int):
    """Nodes, weights and D[a, i] = l_i'(r_a) from numpy polynomial routines."""
    PN = L.Legendre.basis(N)
    inner = np.sort(PN.deriv().roots().real)
    r = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (N * (N + 1) * PN(r) ** 2)
    D = np.zeros((N + 1, N + 1))
    for i in range(N + 1):
        others = np.delete(r, i)
        coeffs = P.polyfromroots(others)
        coeffs = coeffs / P.polyval(r[i], coeffs)  # l_i(r_i) = 1
        D[:, i] = P.polyval(r, P.polyder(coeffs))
    return r, w, D


def element_matrices(N: int, h: float):
    """(S_e, M_e) for an affine cube of side h, local index i + Nq(j + Nq k)."""
    r, w, D = gll_np(N)
    W = np.diag(w)
    K1 = D.T @ W @ D
    kron3 = lambda a, b, c: np.kron(a, np.kron(b, c))  # last factor fastest
    S = 0.5 * h * (kron3(W, W, K1) + kron3(W, K1, W) + kron3(K1, W, W))
    M = (0.5 * h) ** 3 * kron3(W, W, W)
    return S, M


def scatter_matrix(ids: np.ndarray, NG: int) -> np.ndarray:
    """Dense Z (N_L x N_G), one unit entry per unmasked row (eq. scatter_def)."""
    Z = np.zeros((ids.size, NG))
    rows = np.nonzero(ids >= 0)[0]
    Z[rows, ids[rows]] = 1.0
    return Z


def assemble(mesh, lam: float, coef=None) -> np.ndarray:
    """Dense A = Z^T blockdiag(c_e S_e + lambda M_e) Z."""
    S, M = element_matrices(mesh.N, mesh.h)
    Np = mesh.Np
    AL = np.zeros((mesh.NL, mesh.NL))
    for e in range(mesh.E):
        c = 1.0 if coef is None else coef[e]
        AL[e * Np:(e + 1) * Np, e * Np:(e + 1) * Np] = c * S + lam * M
    Z = scatter_matrix(mesh.ids, mesh.NG)
    return Z.T @ AL @ Z


def global_coords(mesh):
    """(x, y, z) of every global node of a structured mesh."""
    r, _, _ = gll_np(mesh.N)
    G, N, h = mesh.G, mesh.N, mesh.h
    g = mesh.grid  # grid index of each global node (Dirichlet meshes skip the boundary)
    gx, gy, gz = g % G, (g // G) % G, g // (G * G)

    def coord(t):
        e = np.minimum(t // N, mesh.K - 1)
        i = t - e * N
        return e * h + 0.5 * h * (r[i] + 1.0)

    return coord(gx), coord(gy), coord(gz)


def node_coords(mesh):
    """(x, y, z) of every global node through each element's trilinear map
    x(r) = sum_v X_v (1 + sx r)(1 + sy s)(1 + sz t) / 8 of its corners
    mesh.verts() (general hexahedra; equal to global_coords when unperturbed)."""
    r, _, _ = gll_np(mesh.N)
    Nq, Np = mesh.Nq, mesh.Np
    l = np.arange(Np)
    ri, rj, rk = r[l % Nq], r[(l // Nq) % Nq], r[l // (Nq * Nq)]
    sh = np.empty((Np, 8))
    for v in range(8):
        sx, sy, sz = (1 if v & 1 else -1), (1 if v & 2 else -1), (1 if v & 4 else -1)
        sh[:, v] = (1 + sx * ri) * (1 + sy * rj) * (1 + sz * rk) / 8.0
    X = np.einsum("lv,evd->eld", sh, mesh.verts())
    ids = mesh.ids.reshape(mesh.E, Np)
    keep = ids >= 0
    out = np.zeros((mesh.NG, 3))
    out[ids[keep]] = X[keep]
    return out[:, 0], out[:, 1], out[:, 2]
