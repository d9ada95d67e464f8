"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the method: it only draws random vectors
and builds the structured-mesh local-to-global maps that both the GPU library
and the CPU oracle take as *inputs*.  Everything is counter-based, so a value
depends only on (seed, stream, index) and never on numpy's generator streams.

Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Value i of stream s under seed S is
``mix(base(S, s) + (i + 1) * GAMMA)`` with ``base = mix(S * GAMMA ^ s * SALT)``.
uniform[-1, 1) = 2 * ((u >> 11) * 2^-53) - 1.  Normals by Box-Muller.

Meshes (the paper's BS6/BS7 workload, Sec. 6.2): structured K x K x K hex
meshes of the unit cube with degree-N GLL nodes; element e = ex + K(ey + K ez),
local node (i, j, k) -> i + Nq (j + Nq k), global node
(ex N + i) + G((ey N + j) + G(ez N + k)) with G = K N + 1.  Element storage
order is a seeded permutation (slot s holds element perm[s]); the global
numbering is unchanged.  Nothing downstream may exploit this structure.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_SALT = np.uint64(0xD1B54A32D192ED03)


def _mix(z):
    z = z.copy() if isinstance(z, np.ndarray) else np.uint64(z)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _base(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GAMMA ^ np.uint64(stream & 0xFFFFFFFF) * _SALT
    return _mix(np.array([s], dtype=np.uint64))[0]


def bits(n: int, seed: int, stream: int = 0, start: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """n raw 64-bit splitmix64 outputs, indices start..start+n-1."""
    out = np.empty(int(n), dtype=np.uint64)
    b = _base(seed, stream)
    for lo in range(0, int(n), chunk):
        hi = min(int(n), lo + chunk)
        i = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = b + i * GAMMA
        out[lo:hi] = _mix(z)
    return out


def uniform(n: int, seed: int, stream: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n float64 values uniform in [lo, hi) (default [-1, 1))."""
    out = np.empty(int(n), dtype=np.float64)
    b = _base(seed, stream)
    chunk = 1 << 24
    for s in range(0, int(n), chunk):
        e = min(int(n), s + chunk)
        i = np.arange(s + 1, e + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = _mix(b + i * GAMMA)
        u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        out[s:e] = lo + (hi - lo) * u
    return out


def normal(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """n standard normals by Box-Muller from two uniform(0,1] streams."""
    u1 = 1.0 - uniform(n, seed, 2 * stream + 1, 0.0, 1.0)  # (0, 1]
    u2 = uniform(n, seed, 2 * stream + 2, 0.0, 1.0)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def lognormal(n: int, seed: int, sigma: float = 1.0, stream: int = 0) -> np.ndarray:
    """n values exp(sigma * g), g standard normal."""
    return np.exp(sigma * normal(n, seed, stream))


def permutation(n: int, seed: int, stream: int = 99) -> np.ndarray:
    """A seeded permutation of range(n): stable argsort of 64-bit keys."""
    return np.argsort(bits(n, seed, stream), kind="stable").astype(np.int64)


class Mesh:
    """Structured K^3 hex mesh of the unit cube, degree N, permuted elements.

    Attributes: K, N, Nq, Np, E, NL, NG, h, ids (int32[NL]), perm (int64[E]),
    grid (int64[NG]: the lexicographic grid index (gx + G (gy + G gz)) of each
    global node).  dirichlet=True masks every local copy of a node on the
    cube's boundary (id -1) and numbers the (G-2)^3 interior nodes
    lexicographically, so that A is the operator with homogeneous Dirichlet
    conditions.  perturb = delta > 0 moves every interior vertex of the
    (K+1)^3 vertex grid by delta h times a seeded uniform[-1, 1) in each
    coordinate (the cube's boundary vertices stay), giving general trilinear
    hexahedra: verts() returns their corners (delta < 0.25 keeps every
    Jacobian positive).
    """

    def __init__(self, K: int, N: int, seed: int | None = 1, permute: bool = True,
                 dirichlet: bool = False, perturb: float = 0.0):
        self.K, self.N = int(K), int(N)
        self.Nq = self.N + 1
        self.Np = self.Nq ** 3
        self.E = self.K ** 3
        self.NL = self.E * self.Np
        self.G = self.K * self.N + 1
        self.NG = self.G ** 3
        self.h = 1.0 / self.K
        self.perturb = float(perturb)
        self.seed = seed
        if self.NL >= 2 ** 31 or self.NG >= 2 ** 31:
            raise ValueError("mesh too large for int32 indices")
        if permute and seed is not None:
            self.perm = permutation(self.E, seed)
        else:
            self.perm = np.arange(self.E, dtype=np.int64)
        self.ids = self._build_ids()
        self.dirichlet = bool(dirichlet)
        if self.dirichlet:
            G = self.G
            g = np.arange(self.NG, dtype=np.int64)
            gx, gy, gz = g % G, (g // G) % G, g // (G * G)
            inner = (gx > 0) & (gx < G - 1) & (gy > 0) & (gy < G - 1) & (gz > 0) & (gz < G - 1)
            new = np.full(self.NG, -1, dtype=np.int64)
            new[inner] = np.arange(int(inner.sum()), dtype=np.int64)
            self.grid = g[inner]
            self.ids = new[self.ids].astype(np.int32)
            self.NG = int(inner.sum())
        else:
            self.grid = np.arange(self.NG, dtype=np.int64)

    def verts(self) -> np.ndarray:
        """Corners [E, 8, 3] of the elements in storage order: corner
        v = vx + 2 (vy + 2 vz) of the element in slot s sits at grid vertex
        (ex + vx, ey + vy, ez + vz) of element perm[s], possibly perturbed."""
        K, h = self.K, self.h
        n1 = K + 1
        g = np.arange(n1 ** 3, dtype=np.int64)
        gv = np.stack([g % n1, (g // n1) % n1, g // (n1 * n1)], axis=1)
        pos = gv.astype(np.float64) * h
        if self.perturb > 0.0:
            inner = np.all((gv > 0) & (gv < K), axis=1)
            seed = 0 if self.seed is None else int(self.seed)
            for d in range(3):
                off = uniform(n1 ** 3, seed, 11 + d) * (self.perturb * h)
                pos[:, d] = np.where(inner, pos[:, d] + off, pos[:, d])
        ex, ey, ez = self.element_coords(self.perm)
        out = np.empty((self.E, 8, 3))
        for v in range(8):
            vx, vy, vz = v & 1, (v >> 1) & 1, (v >> 2) & 1
            out[:, v, :] = pos[(ex + vx) + n1 * ((ey + vy) + n1 * (ez + vz))]
        return out

    def element_coords(self, e):
        """(ex, ey, ez) of natural element index e."""
        K = self.K
        e = np.asarray(e, dtype=np.int64)
        return e % K, (e // K) % K, e // (K * K)

    def _build_ids(self) -> np.ndarray:
        N, Nq, G = self.N, self.Nq, self.G
        a = np.arange(Nq, dtype=np.int64)
        # local offsets of node (i, j, k) relative to the element's corner node
        off = (a[None, None, :] + G * (a[None, :, None] + G * a[:, None, None])).reshape(-1)
        ex, ey, ez = self.element_coords(self.perm)
        corner = ex * N + G * (ey * N + G * (ez * N))
        ids = np.empty(self.NL, dtype=np.int32)
        chunk = max(1, (1 << 24) // self.Np)
        for s in range(0, self.E, chunk):
            e = min(self.E, s + chunk)
            ids[s * self.Np:e * self.Np] = (corner[s:e, None] + off[None, :]).reshape(-1)
        return ids


def batched_specs(nsolves: int = 256, seed: int = 7, nmin: int = 2, nmax: int = 8,
                  kmin: int = 4, kmax: int = 24):
    """(N, K) per solve: N uniform in {nmin..nmax}, K uniform in {kmin..kmax}."""
    u = bits(2 * nsolves, seed, stream=1234)
    Ns = nmin + (u[:nsolves] % np.uint64(nmax - nmin + 1)).astype(np.int64)
    Ks = kmin + (u[nsolves:] % np.uint64(kmax - kmin + 1)).astype(np.int64)
    return [(int(n), int(k)) for n, k in zip(Ns, Ks)]
