"""FP64 CPU oracle for the Benchmark Streaming operations and CG.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` leg are the only callers.
The GPU library never imports, links or executes anything in this directory,
and this directory imports nothing from the GPU package.

``bs_oracle.c`` holds the definitions (Table 1 BS1-BS7, eq. scatter_def,
eqs. global_system / assembled_stiff / assembled_mass, Algorithm 1); this
module only compiles it with gcc and marshals numpy arrays through ctypes.
``bs_oracle_omp.c`` spreads the same plain BS loops over the host cores
(OpenMP), only to time a multi-core CPU baseline (``Omp``).

Parity is pinned for every routine here by ``tests/test_oracle_pins.py``
(closed forms, invariants, brute force and exact rational arithmetic).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbs_oracle.so")
_SOURCES = ["bs_oracle.c", "mlp_oracle.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FP contraction, no fast-math."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_OMP_LIB_PATH = os.path.join(_BUILD, "libbs_oracle_omp.so")
_omp_lib = None


def build_omp(force: bool = False) -> str:
    """Compile bs_oracle_omp.c (the plain BS loops over the host cores) with
    gcc -fopenmp, same floating-point flags as the oracle."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "bs_oracle_omp.c")
    if not force and os.path.exists(_OMP_LIB_PATH) and \
            os.path.getmtime(_OMP_LIB_PATH) >= os.path.getmtime(src):
        return _OMP_LIB_PATH
    tmp = _OMP_LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OMP_LIB_PATH)
    return _OMP_LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double

_SIGS = {
    "bso_copy": (None, [_i64, _D, _D]),
    "bso_axpy": (None, [_i64, _dbl, _D, _dbl, _D]),
    "bso_norm": (None, [_i64, _D, _D]),
    "bso_dot": (_dbl, [_i64, _D, _D]),
    "bso_cg_update": (_dbl, [_i64, _dbl, _D, _D, _D, _D]),
    "bso_scatter": (None, [_i64, _I, _D, _D]),
    "bso_gather": (None, [_i64, _i64, _I, _D, _D]),
    "bso_valence": (None, [_i64, _i64, _I, _I]),
    "bso_gll": (_int, [_int, _D, _D, _D]),
    "bso_csr": (None, [_i64, _i64, _I, _I, _I]),
    "bso_axpy_f32": (None, [_i64, ctypes.c_float, _F, ctypes.c_float, _F]),
    "bso_dot_f32": (_dbl, [_i64, _F, _F]),
    "bso_cg_update_f32": (_dbl, [_i64, ctypes.c_float, _F, _F, _F, _F]),
    "bso_scatter_f32": (None, [_i64, _I, _F, _F]),
    "bso_gather_f32": (None, [_i64, _i64, _I, _F, _F]),
    "bso_apply_A": (_int, [_int, _int, _dbl, _dbl, _D, _I, _i64, _D, _D]),
    "bso_apply_local": (_int, [_int, _int, _dbl, _dbl, _D, _D, _D]),
    "bso_diag_A": (_int, [_int, _int, _dbl, _dbl, _D, _I, _i64, _D]),
    "bso_cg": (_int, [_int, _int, _dbl, _dbl, _D, _I, _i64, _D, _D, _dbl, _int, _int,
                      _D, _D, _D]),
    "bso_pcg_jacobi": (_int, [_int, _int, _dbl, _dbl, _D, _I, _i64, _D, _D, _dbl, _int, _D]),
    "bso_pcg_block_jacobi": (_int, [_int, _int, _dbl, _dbl, _D, _I, _i64, _D, _D, _dbl, _int,
                                    _D]),
    "bso_apply_A_geo": (_int, [_int, _int, _dbl, _D, _D, _I, _i64, _D, _D]),
    "bso_apply_local_geo": (_int, [_int, _int, _dbl, _D, _D, _D, _D]),
    "bso_diag_A_geo": (_int, [_int, _int, _dbl, _D, _D, _I, _i64, _D]),
    "bso_cg_geo": (_int, [_int, _int, _dbl, _D, _D, _I, _i64, _D, _D, _dbl, _int, _int,
                          _D, _D, _D]),
    "bso_pcg_jacobi_geo": (_int, [_int, _int, _dbl, _D, _D, _I, _i64, _D, _D, _dbl, _int,
                                  _D]),
    "bso_cg_ir_f32": (_int, [_int, _int, _dbl, _dbl, _D, _I, _i64, _D, _D, _dbl, _int,
                             _dbl, _int, ctypes.POINTER(_int), _D]),
}


def lib():
    """Build (if stale) and load the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def omp_lib():
    """Build (if stale) and load the OpenMP build of the plain BS loops."""
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            L = ctypes.CDLL(build_omp())
            sigs = {"bso_omp_threads": (_int, []),
                    "bso_omp_copy": (None, [_i64, _D, _D]),
                    "bso_omp_axpy": (None, [_i64, _dbl, _D, _dbl, _D]),
                    "bso_omp_norm": (None, [_i64, _D, _D]),
                    "bso_omp_dot": (_dbl, [_i64, _D, _D]),
                    "bso_omp_cg_update": (_dbl, [_i64, _dbl, _D, _D, _D, _D]),
                    "bso_omp_scatter": (None, [_i64, _I, _D, _D]),
                    "bso_omp_gather_csr": (None, [_i64, _I, _I, _D, _D])}
            for name, (res, args) in sigs.items():
                fn = getattr(L, name)
                fn.restype, fn.argtypes = res, args
            _omp_lib = L
    return _omp_lib


class Omp:
    """The plain BS1-BS7 loops over all host cores (bs_oracle_omp.c); in
    place on the caller's arrays, for timing.  gather() needs the CSR of
    Z^T, built once from the map (csr())."""

    def __init__(self):
        self.L = omp_lib()
        self.threads = self.L.bso_omp_threads()

    def copy(self, x, y):
        self.L.bso_omp_copy(x.size, _d(x), _d(y))

    def axpy(self, alpha, x, beta, y):
        self.L.bso_omp_axpy(x.size, alpha, _d(x), beta, _d(y))

    def norm(self, x):
        out = np.empty(2)
        self.L.bso_omp_norm(x.size, _d(x), _d(out))
        return out

    def dot(self, x, y):
        return self.L.bso_omp_dot(x.size, _d(x), _d(y))

    def cg_update(self, alpha, p, Ap, x, r):
        return self.L.bso_omp_cg_update(x.size, alpha, _d(p), _d(Ap), _d(x), _d(r))

    def scatter(self, ids, qG, qL):
        self.L.bso_omp_scatter(ids.size, _i(ids), _d(qG), _d(qL))

    def gather(self, row_starts, col_ids, qL, qG):
        self.L.bso_omp_gather_csr(qG.size, _i(row_starts), _i(col_ids), _d(qL), _d(qG))


def _d(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ids(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- BS1-BS5

def copy(x):
    """BS1 (Table 1): y = x."""
    x = _f64(x)
    y = np.empty_like(x)
    lib().bso_copy(x.size, _d(x), _d(y))
    return y


def axpy(alpha, x, beta, y):
    """BS2 (Table 1): returns fma(alpha, x, beta*y)."""
    x = _f64(x)
    y = _f64(y).copy()
    lib().bso_axpy(x.size, float(alpha), _d(x), float(beta), _d(y))
    return y


def norm(x):
    """BS3 (Table 1): returns (x.x, sqrt(x.x))."""
    x = _f64(x)
    out = np.zeros(2)
    lib().bso_norm(x.size, _d(x), _d(out))
    return float(out[0]), float(out[1])


def dot(x, y):
    """BS4 (Table 1): x.y."""
    x, y = _f64(x), _f64(y)
    return float(lib().bso_dot(x.size, _d(x), _d(y)))


def cg_update(alpha, p, Ap, x, r):
    """BS5 (Table 1, Algorithm 1 steps 8-10): returns (x', r', r'.r')."""
    p, Ap = _f64(p), _f64(Ap)
    x, r = _f64(x).copy(), _f64(r).copy()
    rr = lib().bso_cg_update(x.size, float(alpha), _d(p), _d(Ap), _d(x), _d(r))
    return x, r, float(rr)


# ---------------------------------------------------------------- BS6/BS7

def scatter(ids, qG, qL_init):
    """BS7 (eq. scatter_def): q_L = Z q_G, masked entries keep qL_init."""
    ids, qG = _ids(ids), _f64(qG)
    qL = _f64(qL_init).copy()
    lib().bso_scatter(ids.size, _i(ids), _d(qG), _d(qL))
    return qL


def gather(ids, qL, NG):
    """BS6 (eq. scatter_def): q_G = Z^T q_L, ascending local order."""
    ids, qL = _ids(ids), _f64(qL)
    qG = np.empty(int(NG))
    lib().bso_gather(ids.size, int(NG), _i(ids), _d(qL), _d(qG))
    return qG


def valence(ids, NG):
    """diag(Z^T Z): the number of local copies of every global node."""
    ids = _ids(ids)
    v = np.empty(int(NG), dtype=np.int32)
    lib().bso_valence(ids.size, int(NG), _i(ids), _i(v))
    return v


def csr(ids, NG):
    """CSR of Z^T by definition: (rowStarts[NG+1], colIds ascending per row)."""
    ids = _ids(ids)
    rs = np.empty(int(NG) + 1, dtype=np.int32)
    ci = np.empty(max(int((ids >= 0).sum()), 1), dtype=np.int32)
    lib().bso_csr(ids.size, int(NG), _i(ids), _i(rs), _i(ci))
    return rs, ci[:int((ids >= 0).sum())]


# ---------------------------------------------------------------- FP32 twins

def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fp(a):
    return a.ctypes.data_as(_F)


def axpy_f32(alpha, x, beta, y):
    """BS2 in float: fmaf(alpha, x, beta*y)."""
    x, y = _f32(x), _f32(y).copy()
    lib().bso_axpy_f32(x.size, float(alpha), _fp(x), float(beta), _fp(y))
    return y


def dot_f32(x, y):
    """Sum of products of float vectors, exact products, Dot2 summation."""
    x, y = _f32(x), _f32(y)
    return float(lib().bso_dot_f32(x.size, _fp(x), _fp(y)))


def cg_update_f32(alpha, p, Ap, x, r):
    """BS5 in float; returns (x', r', r'.r')."""
    p, Ap, x, r = _f32(p), _f32(Ap), _f32(x).copy(), _f32(r).copy()
    rr = lib().bso_cg_update_f32(x.size, float(alpha), _fp(p), _fp(Ap), _fp(x), _fp(r))
    return x, r, float(rr)


def scatter_f32(ids, qG, qL_init):
    ids, qG, qL = _ids(ids), _f32(qG), _f32(qL_init).copy()
    lib().bso_scatter_f32(ids.size, _i(ids), _fp(qG), _fp(qL))
    return qL


def gather_f32(ids, qL, NG):
    ids, qL = _ids(ids), _f32(qL)
    qG = np.empty(int(NG), dtype=np.float32)
    lib().bso_gather_f32(ids.size, int(NG), _i(ids), _fp(qL), _fp(qG))
    return qG


# ---------------------------------------------------------------- operator

def gll(N):
    """GLL nodes r, weights w and D[a, i] = l_i'(r_a) (Sec. 2, eq. basis)."""
    r, w, D = np.zeros(N + 1), np.zeros(N + 1), np.zeros((N + 1) * (N + 1))
    if lib().bso_gll(int(N), _d(r), _d(w), _d(D)):
        raise ValueError(f"unsupported degree {N}")
    return r, w, D.reshape(N + 1, N + 1)


def _coef(coef):
    return None if coef is None else _f64(coef)


def apply_A(E, N, h, lam, ids, NG, p, coef=None):
    """A p with A = Z^T (c S_L + lambda M_L) Z (eqs. global_system,
    assembled_stiff, assembled_mass)."""
    ids, p, coef = _ids(ids), _f64(p), _coef(coef)
    Ap = np.empty(int(NG))
    rc = lib().bso_apply_A(E, N, float(h), float(lam), _d(coef), _i(ids), int(NG), _d(p), _d(Ap))
    if rc:
        raise RuntimeError(f"bso_apply_A failed ({rc})")
    return Ap


def apply_local(E, N, h, lam, uL, coef=None):
    """Block-diagonal A_L u_L (no Z, no Z^T)."""
    uL, coef = _f64(uL), _coef(coef)
    out = np.empty_like(uL)
    rc = lib().bso_apply_local(E, N, float(h), float(lam), _d(coef), _d(uL), _d(out))
    if rc:
        raise RuntimeError(f"bso_apply_local failed ({rc})")
    return out


def diag_A(E, N, h, lam, ids, NG, coef=None):
    """diag(A) = Z^T diag(A_L)."""
    ids, coef = _ids(ids), _coef(coef)
    d = np.empty(int(NG))
    rc = lib().bso_diag_A(E, N, float(h), float(lam), _d(coef), _i(ids), int(NG), _d(d))
    if rc:
        raise RuntimeError(f"bso_diag_A failed ({rc})")
    return d


def cg(E, N, h, lam, ids, NG, b, x0=None, tol=1e-8, maxit=1000, fixed_iters=False, coef=None):
    """Algorithm 1.  Returns (x, iters, alpha[], beta[], rr[])."""
    ids, b, coef = _ids(ids), _f64(b), _coef(coef)
    x = np.zeros(int(NG)) if x0 is None else _f64(x0).copy()
    ha, hb, hr = np.zeros(maxit + 1), np.zeros(maxit + 1), np.zeros(maxit + 2)
    it = lib().bso_cg(E, N, float(h), float(lam), _d(coef), _i(ids), int(NG), _d(b), _d(x),
                      float(tol), int(maxit), int(bool(fixed_iters)), _d(ha), _d(hb), _d(hr))
    if it < 0:
        raise RuntimeError(f"bso_cg failed ({it})")
    return x, it, ha[:it], hb[:it], hr[:it + 1]


def pcg_jacobi(E, N, h, lam, ids, NG, b, tol=1e-8, maxit=1000, coef=None):
    """Jacobi-preconditioned CG.  Returns (x, iters, rr[])."""
    ids, b, coef = _ids(ids), _f64(b), _coef(coef)
    x = np.zeros(int(NG))
    hr = np.zeros(maxit + 2)
    it = lib().bso_pcg_jacobi(E, N, float(h), float(lam), _d(coef), _i(ids), int(NG), _d(b),
                              _d(x), float(tol), int(maxit), _d(hr))
    if it < 0:
        raise RuntimeError(f"bso_pcg_jacobi failed ({it})")
    return x, it, hr[:it + 1]


# ---------------------------------------------------------------- general hexahedra
# verts: float64 [E, 8, 3], corner v = vx + 2 (vy + 2 vz) of element e (the
# trilinear map of bs_oracle.c); the operator is the same weak form with the
# non-affine geometric factors w det J J^-1 J^-T at every GLL node.

def pcg_block_jacobi(E, N, h, lam, ids, NG, b, tol=1e-8, maxit=1000, coef=None):
    """PCG with the element-interior blocks solved exactly (Cholesky) and
    Jacobi elsewhere.  Returns (x, iters, rr[])."""
    ids, b, coef = _ids(ids), _f64(b), _coef(coef)
    x = np.zeros(int(NG))
    hr = np.zeros(maxit + 1)
    it = lib().bso_pcg_block_jacobi(E, N, float(h), float(lam), _d(coef), _i(ids), int(NG),
                                    _d(b), _d(x), float(tol), int(maxit), _d(hr))
    if it < 0:
        raise RuntimeError(f"bso_pcg_block_jacobi failed ({it})")
    return x, it, hr[:it + 1]


def _verts(verts, E):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    if v.size != 24 * E:
        raise ValueError("verts must hold 8 corners x 3 coordinates per element")
    return v


def apply_A_geo(E, N, lam, verts, ids, NG, p, coef=None):
    ids, p, coef, v = _ids(ids), _f64(p), _coef(coef), _verts(verts, E)
    Ap = np.empty(int(NG))
    rc = lib().bso_apply_A_geo(E, N, float(lam), _d(coef), _d(v), _i(ids), int(NG), _d(p),
                               _d(Ap))
    if rc:
        raise RuntimeError(f"bso_apply_A_geo failed ({rc})")
    return Ap


def apply_local_geo(E, N, lam, verts, uL, coef=None):
    uL, coef, v = _f64(uL), _coef(coef), _verts(verts, E)
    out = np.empty_like(uL)
    rc = lib().bso_apply_local_geo(E, N, float(lam), _d(coef), _d(v), _d(uL), _d(out))
    if rc:
        raise RuntimeError(f"bso_apply_local_geo failed ({rc})")
    return out


def diag_A_geo(E, N, lam, verts, ids, NG, coef=None):
    ids, coef, v = _ids(ids), _coef(coef), _verts(verts, E)
    d = np.empty(int(NG))
    rc = lib().bso_diag_A_geo(E, N, float(lam), _d(coef), _d(v), _i(ids), int(NG), _d(d))
    if rc:
        raise RuntimeError(f"bso_diag_A_geo failed ({rc})")
    return d


def cg_geo(E, N, lam, verts, ids, NG, b, tol=1e-8, maxit=1000, fixed_iters=False, coef=None):
    """Algorithm 1 on the general-hexahedron operator.  (x, iters, alpha, beta, rr)."""
    ids, b, coef, v = _ids(ids), _f64(b), _coef(coef), _verts(verts, E)
    x = np.zeros(int(NG))
    ha, hb, hr = np.zeros(maxit + 1), np.zeros(maxit + 1), np.zeros(maxit + 2)
    it = lib().bso_cg_geo(E, N, float(lam), _d(coef), _d(v), _i(ids), int(NG), _d(b), _d(x),
                          float(tol), int(maxit), int(bool(fixed_iters)), _d(ha), _d(hb),
                          _d(hr))
    if it < 0:
        raise RuntimeError(f"bso_cg_geo failed ({it})")
    return x, it, ha[:it], hb[:it], hr[:it + 1]


def pcg_jacobi_geo(E, N, lam, verts, ids, NG, b, tol=1e-8, maxit=1000, coef=None):
    ids, b, coef, v = _ids(ids), _f64(b), _coef(coef), _verts(verts, E)
    x = np.zeros(int(NG))
    hr = np.zeros(maxit + 2)
    it = lib().bso_pcg_jacobi_geo(E, N, float(lam), _d(coef), _d(v), _i(ids), int(NG), _d(b),
                                  _d(x), float(tol), int(maxit), _d(hr))
    if it < 0:
        raise RuntimeError(f"bso_pcg_jacobi_geo failed ({it})")
    return x, it, hr[:it + 1]


def cg_ir_f32(E, N, h, lam, ids, NG, b, outer_tol=1e-10, outer_maxit=50, inner_tol=1e-4,
              inner_maxit=2000, coef=None):
    """FP32-storage CG inside an FP64 iterative-refinement loop.
    Returns (x, inner_iters, outer_iters, true_relres)."""
    ids, b, coef = _ids(ids), _f64(b), _coef(coef)
    x = np.zeros(int(NG))
    outer = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    it = lib().bso_cg_ir_f32(E, N, float(h), float(lam), _d(coef), _i(ids), int(NG), _d(b),
                             _d(x), float(outer_tol), int(outer_maxit), float(inner_tol),
                             int(inner_maxit), ctypes.byref(outer), ctypes.byref(rel))
    if it < 0:
        raise RuntimeError(f"bso_cg_ir_f32 failed ({it})")
    return x, it, outer.value, rel.value


# ---------------------------------------------------------------- learned preconditioner

_SIGS.update({
    "bso_bf16_round": (None, [_i64, _F, _F]),
    "bso_mlp_forward": (None, [_i64, _int, _int, _F, _F, _F, _D, _D, _int, _int]),
    "bso_mlp_loss_grad": (_dbl, [_i64, _int, _int, _F, _F, _F, _F, _D, _D, _int]),
    "bso_adam": (None, [_i64, _F, _F, _F, _F, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                        ctypes.c_float, _int]),
    "bso_fpcg": (_int, [_int, _int, _dbl, _dbl, _D, _I, _i64, _F, _F, _int, _int, _int, _D, _D,
                        _dbl, _int, _D, ctypes.POINTER(_int)]),
    "bso_interior_pairs": (_int, [_int, _int, _dbl, _dbl, _D, _I, _i64, _D, _i64, _I, _int, _F,
                                  _F]),
    "bso_fpcg_judged": (_int, [_int, _int, _dbl, _dbl, _D, _I, _i64, _F, _F, _int, _int, _int,
                               _D, _D, _dbl, _int, _int, _int, _D, ctypes.POINTER(_int),
                               ctypes.POINTER(_int)]),
})


def _lib_mlp():
    L = lib()
    for name in ("bso_bf16_round", "bso_mlp_forward", "bso_mlp_loss_grad", "bso_adam", "bso_fpcg",
                 "bso_interior_pairs", "bso_fpcg_judged"):
        res, args = _SIGS[name]
        fn = getattr(L, name)
        fn.restype, fn.argtypes = res, args
    return L


def bf16_round(a):
    """Round float values to bfloat16 (nearest even), returned as float32."""
    a = _f32(a)
    out = np.empty_like(a)
    _lib_mlp().bso_bf16_round(a.size, _fp(a), _fp(out))
    return out


PREC_FP64, PREC_BF16, PREC_BF16X3 = 0, 1, 2


def mlp_forward(W1, W2, X, prec=PREC_FP64, odd=False):
    """y = W2 relu(W1 x) per row of X (W1: H x D, W2: D x H), or its odd part
    (f(x) - f(-x)) / 2 when odd.  prec: PREC_FP64, PREC_BF16 or PREC_BF16X3.
    Returns (Y, hidden of f(x))."""
    W1, W2, X = _f32(W1), _f32(W2), _f32(X)
    H, D = W1.shape
    B = X.shape[0]
    Y, hid = np.empty((B, D)), np.empty((B, H))
    _lib_mlp().bso_mlp_forward(B, D, H, _fp(W1), _fp(W2), _fp(X), _d(Y), _d(hid), int(prec),
                               int(bool(odd)))
    return Y, hid


def mlp_loss_grad(W1, W2, X, T, prec=PREC_FP64):
    """MSE loss and (dL/dW1, dL/dW2) in FP64 (forward in mode prec)."""
    W1, W2, X, T = _f32(W1), _f32(W2), _f32(X), _f32(T)
    H, D = W1.shape
    g1, g2 = np.empty((H, D)), np.empty((D, H))
    loss = _lib_mlp().bso_mlp_loss_grad(X.shape[0], D, H, _fp(W1), _fp(W2), _fp(X), _fp(T),
                                        _d(g1), _d(g2), int(prec))
    return float(loss), g1, g2


def adam(w, g, m, v, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in float, in place on copies; returns (w, m, v)."""
    w, g, m, v = _f32(w).copy(), _f32(g), _f32(m).copy(), _f32(v).copy()
    _lib_mlp().bso_adam(w.size, _fp(w), _fp(g), _fp(m), _fp(v), lr, b1, b2, eps, int(t))
    return w, m, v


def fpcg(E, N, h, lam, ids, NG, b, W1=None, W2=None, prec=PREC_BF16, odd=False, tol=1e-8,
         maxit=10000, coef=None):
    """Flexible PCG with the learned correction (W2 None: Jacobi only).
    Returns (x, iters, rr[], fallbacks)."""
    ids, b, coef = _ids(ids), _f64(b), _coef(coef)
    x = np.zeros(int(NG))
    hr = np.zeros(maxit + 2)
    fb = ctypes.c_int(0)
    H = 0 if W1 is None else int(np.asarray(W1).shape[0])
    W1p = None if W1 is None else _f32(W1)
    W2p = None if W2 is None else _f32(W2)
    it = _lib_mlp().bso_fpcg(E, N, float(h), float(lam), _d(coef), _i(ids), int(NG),
                             None if W1p is None else _fp(W1p),
                             None if W2p is None else _fp(W2p), H, int(prec), int(bool(odd)),
                             _d(b), _d(x), float(tol), int(maxit), _d(hr), ctypes.byref(fb))
    if it < 0:
        raise RuntimeError(f"bso_fpcg failed ({it})")
    return x, it, hr[:it + 1], fb.value


def judge_stall(NG):
    """The Jacobi judge's patience: max(1024, 16 N_G^(1/3)) iterations."""
    return max(1024, int(16.0 * float(NG) ** (1.0 / 3.0)))


def fpcg_judged(E, N, h, lam, ids, NG, b, W1, W2, prec=PREC_BF16, odd=False, tol=1e-8,
                maxit=10000, coef=None, period=8, stall=None):
    """Flexible PCG with the learned correction and the Jacobi judge checked
    every `period` iterations (patience `stall`, default judge_stall(NG)).
    Returns (x, iters, rr[], fallbacks, switched_at)."""
    ids, b, coef = _ids(ids), _f64(b), _coef(coef)
    x = np.zeros(int(NG))
    hr = np.zeros(maxit + 2)
    fb, sw = ctypes.c_int(0), ctypes.c_int(0)
    W1p, W2p = _f32(W1), _f32(W2)
    stall = judge_stall(NG) if stall is None else int(stall)
    it = _lib_mlp().bso_fpcg_judged(E, N, float(h), float(lam), _d(coef), _i(ids), int(NG),
                                    _fp(W1p), _fp(W2p), int(W1p.shape[0]), int(prec),
                                    int(bool(odd)), _d(b), _d(x), float(tol), int(maxit),
                                    int(period), stall, _d(hr), ctypes.byref(fb),
                                    ctypes.byref(sw))
    if it < 0:
        raise RuntimeError(f"bso_fpcg_judged failed ({it})")
    return x, it, hr[:it + 1], fb.value, sw.value


def interior_pairs(E, N, h, lam, ids, NG, r, elems, negate_odd=False, coef=None):
    """Training pairs (X, T), each [len(elems) x (N+1)^3] float32: X = s u / rms,
    T = s (A_II^-1 r_I - u_I) / rms on interior nodes (0 elsewhere), u = D^-1 r."""
    ids, r, coef = _ids(ids), _f64(r), _coef(coef)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    Np = (N + 1) ** 3
    X = np.zeros((len(elems), Np), np.float32)
    T = np.zeros((len(elems), Np), np.float32)
    rc = _lib_mlp().bso_interior_pairs(E, N, float(h), float(lam), _d(coef), _i(ids), int(NG),
                                       _d(r), len(elems), _i(elems), int(bool(negate_odd)),
                                       _fp(X), _fp(T))
    if rc:
        raise RuntimeError(f"bso_interior_pairs failed ({rc})")
    return X, T
