"""Thin Python binding of libbs (include/bs.h) over torch CUDA tensors.

Argument marshalling only: every step runs in the library's CUDA kernels.
Tensors must be contiguous CUDA tensors on the current device; calls are
enqueued on torch's current stream.  There is no CPU fallback: if libbs.so
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

BS_OK = 0
BS_ERR_ARG = 1
BS_ERR_CUDA = 2
BS_ERR_TIMEOUT = 3
BS_ERR_BREAKDOWN = 4
BS_ERR_NOT_CONVERGED = 5
BS_ERR_DEVICE_CHECK = 6
BS_ERR_ALLOC = 7

BS_CG_FIXED_ITERS = 1
BS_CG_JACOBI = 2
BS_CG_GRAPH = 4
BS_CG_X0 = 8
BS_CG_REFINED_F32 = 32
BS_CG_FF_OPERATOR = 256
BS_CG_SCATTERED = 512
BS_CG_BLOCK_JACOBI = 1024
BS_OP_FUSED = 1
BS_OP_DIRECT = 2
BS_MLP_BF16X3 = 1
BS_MLP_ODD = 2
BS_FPCG_ODD = 64
BS_FPCG_NO_JUDGE = 128


class BSError(RuntimeError):
    def __init__(self, status, fn, detail):
        super().__init__(f"{fn}: status {status} ({detail})")
        self.status = status


class CgInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("status", ctypes.c_int32),
                ("outer", ctypes.c_int32), ("fallbacks", ctypes.c_int32),
                ("rr", ctypes.c_double), ("bb", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_d = ctypes.c_double
_f = ctypes.c_float
_pp = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "bs_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "bs_last_error": (ctypes.c_char_p, []),
    "bs_version": (ctypes.c_int, []),
    "bs_check_enabled": (ctypes.c_int, []),
    "bs_check_device": (ctypes.c_int, []),
    "bs_workspace_create": (ctypes.c_int, [_pp]),
    "bs_workspace_destroy": (ctypes.c_int, [_vp]),
    "bs_copy": (ctypes.c_int, [_i64, _vp, _vp, _vp]),
    "bs_axpy": (ctypes.c_int, [_i64, _d, _vp, _d, _vp, _vp]),
    "bs_norm": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp]),
    "bs_dot": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _vp]),
    "bs_cg_update": (ctypes.c_int, [_i64, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "bs_copy_f32": (ctypes.c_int, [_i64, _vp, _vp, _vp]),
    "bs_axpy_f32": (ctypes.c_int, [_i64, _f, _vp, _f, _vp, _vp]),
    "bs_norm_f32": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp]),
    "bs_dot_f32": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _vp]),
    "bs_cg_update_f32": (ctypes.c_int, [_i64, _f, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "bs_map_create": (ctypes.c_int, [_i32, _i32, _i64, _vp, _pp]),
    "bs_map_destroy": (ctypes.c_int, [_vp]),
    "bs_map_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                   ctypes.POINTER(_i64)]),
    "bs_map_export": (ctypes.c_int, [_vp, _vp, _vp]),
    "bs_map_valence": (ctypes.c_int, [_vp, _vp, _vp]),
    "bs_scatter": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bs_gather": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bs_scatter_f32": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bs_gather_f32": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bs_problem_create": (ctypes.c_int, [_vp, _d, _d, _vp, _pp]),
    "bs_problem_create_geo": (ctypes.c_int, [_vp, _d, _vp, _vp, _pp]),
    "bs_problem_destroy": (ctypes.c_int, [_vp]),
    "bs_apply_A": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bs_apply_A_ff": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bs_apply_local": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bs_diag_A": (ctypes.c_int, [_vp, _vp, _vp]),
    "bs_cg_solve": (ctypes.c_int, [_vp, _vp, _vp, _d, _i32, _i32, _vp,
                                   ctypes.POINTER(CgInfo), _vp]),
    "bs_cg_solve_refined_f32": (ctypes.c_int, [_vp, _vp, _vp, _d, _i32, _d, _i32, _i32,
                                               ctypes.POINTER(CgInfo), _vp]),
    "bs_cg_solve_batched": (ctypes.c_int, [_i32, _vp, _vp, _vp, _d, _i32, _i32,
                                           ctypes.POINTER(CgInfo), _vp]),
    "bs_operator_mode": (ctypes.c_int, [_i32]),
}


def operator_mode(mode=-1):
    """bs_operator_mode: bits BS_OP_FUSED, BS_OP_DIRECT (0, the default:
    unfused, even-odd element kernels); returns the previous mode (-1: query
    only)."""
    return lib().bs_operator_mode(int(mode))


def operator_fusion(on=-1):
    """Set (1) or clear (0) BS_OP_FUSED, keeping the other bits; returns the
    previous state of the bit (-1: query only)."""
    prev = operator_mode(-1)
    if on >= 0:
        operator_mode((prev & ~BS_OP_FUSED) | (BS_OP_FUSED if on else 0))
    return 1 if prev & BS_OP_FUSED else 0


def checked() -> bool:
    """True when the environment sets BS_CHECK (not 0): the checked build
    (-DBS_CHECK=1, every index read from memory tested on the device) is
    loaded, and every call is followed by bs_check_device."""
    return os.environ.get("BS_CHECK", "0") not in ("", "0")


def library_path() -> str:
    return _build.lib_path(check=checked())


# entry points that touch no device state (no check after them)
_NO_DEVICE = {"bs_error_string", "bs_last_error", "bs_version", "bs_check_enabled",
              "bs_check_device"}


def _device_check(result, func, args):
    """ctypes errcheck of the checked build: collect the device-side check
    words after the call and raise on a recorded failure."""
    rc = _lib.bs_check_device()
    if rc != BS_OK:
        raise BSError(rc, func.__name__ + " (device check)",
                      _lib.bs_last_error().decode(errors="replace"))
    return result


def lib():
    """Load libbs.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            chk = checked()
            path = _build.lib_path(check=chk)
            if _build.is_stale(check=chk):
                try:
                    path = _build.build(check=chk)
                except Exception as exc:  # no nvcc or failed build: no fallback
                    if not os.path.exists(path):
                        raise RuntimeError(f"{path} is missing and cannot be built: {exc}")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            if bool(L.bs_check_enabled()) != chk:
                raise RuntimeError(f"{path}: checked build {bool(L.bs_check_enabled())}, "
                                   f"wanted {chk}")
            if chk:
                for name in _SIGS:
                    if name not in _NO_DEVICE:
                        getattr(L, name).errcheck = _device_check
            _lib = L
    return _lib


def _check(rc, fn):
    if rc != BS_OK:
        L = lib()
        raise BSError(rc, fn, L.bs_last_error().decode(errors="replace"))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=torch.float64, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Workspace:
    """Reduction scratch of the current device (bs_workspace)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib().bs_workspace_create(ctypes.byref(h)), "bs_workspace_create")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bs_workspace_destroy(self.handle)
            self.handle = None


_ws = {}


def workspace() -> Workspace:
    """The default workspace of the current device (one per device)."""
    dev = torch.cuda.current_device()
    if dev not in _ws:
        _ws[dev] = Workspace()
    return _ws[dev]


# ---------------------------------------------------------------- BS1-BS5

def _sfx(t):
    return "_f32" if t.dtype == torch.float32 else ""


def copy(x, y=None):
    """BS1: y = x."""
    y = torch.empty_like(x) if y is None else y
    _check(getattr(lib(), "bs_copy" + _sfx(x))(x.numel(), _ptr(x, x.dtype, "x"),
                                               _ptr(y, x.dtype, "y"), _stream()), "bs_copy")
    return y


def axpy(alpha, x, beta, y):
    """BS2: y = fma(alpha, x, beta*y), in place on y."""
    _check(getattr(lib(), "bs_axpy" + _sfx(x))(x.numel(), alpha, _ptr(x, x.dtype, "x"), beta,
                                               _ptr(y, x.dtype, "y"), _stream()), "bs_axpy")
    return y


def norm(x, out=None, ws=None):
    """BS3: device tensor [x.x, sqrt(x.x)] (float64)."""
    out = torch.empty(2, dtype=torch.float64, device=x.device) if out is None else out
    ws = ws or workspace()
    _check(getattr(lib(), "bs_norm" + _sfx(x))(x.numel(), _ptr(x, x.dtype, "x"), _ptr(out),
                                               ws.handle, _stream()), "bs_norm")
    return out


def dot(x, y, out=None, ws=None):
    """BS4: device tensor [x.y] (float64)."""
    out = torch.empty(1, dtype=torch.float64, device=x.device) if out is None else out
    ws = ws or workspace()
    _check(getattr(lib(), "bs_dot" + _sfx(x))(x.numel(), _ptr(x, x.dtype, "x"),
                                              _ptr(y, x.dtype, "y"), _ptr(out), ws.handle,
                                              _stream()), "bs_dot")
    return out


def cg_update(alpha, p, Ap, x, r, out=None, ws=None):
    """BS5: x += alpha p; r -= alpha Ap (in place); device tensor [r.r]."""
    out = torch.empty(1, dtype=torch.float64, device=x.device) if out is None else out
    ws = ws or workspace()
    t = x.dtype
    _check(getattr(lib(), "bs_cg_update" + _sfx(x))(
        x.numel(), alpha, _ptr(p, t, "p"), _ptr(Ap, t, "Ap"), _ptr(x, t, "x"), _ptr(r, t, "r"),
        _ptr(out), ws.handle, _stream()), "bs_cg_update")
    return out


# ---------------------------------------------------------------- BS6/BS7

class Map:
    """The scatter operator Z from an int32 local-to-global map (bs_map)."""

    def __init__(self, E: int, N: int, NG: int, l2g: np.ndarray):
        l2g = np.ascontiguousarray(l2g, dtype=np.int32)
        Np = (N + 1) ** 3
        if l2g.size != E * Np:
            raise ValueError("l2g must have E*(N+1)^3 entries")
        h = ctypes.c_void_p()
        _check(lib().bs_map_create(E, N, NG, l2g.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(h)), "bs_map_create")
        self.handle, self.E, self.N, self.NG, self.NL = h, E, N, NG, E * Np
        nl, ng, nnz = _i64(), _i64(), _i64()
        _check(lib().bs_map_info(h, ctypes.byref(nl), ctypes.byref(ng), ctypes.byref(nnz)),
               "bs_map_info")
        self.nnz = nnz.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bs_map_destroy(self.handle)
            self.handle = None

    def export(self):
        rs = np.empty(self.NG + 1, dtype=np.int32)
        ci = np.empty(max(self.nnz, 1), dtype=np.int32)
        _check(lib().bs_map_export(self.handle, rs.ctypes.data_as(ctypes.c_void_p),
                                   ci.ctypes.data_as(ctypes.c_void_p)), "bs_map_export")
        return rs, ci[:self.nnz]

    def valence(self, device=None):
        out = torch.empty(self.NG, dtype=torch.int32, device=device or "cuda")
        _check(lib().bs_map_valence(self.handle, _ptr(out, torch.int32), _stream()),
               "bs_map_valence")
        return out

    def scatter(self, qG, qL=None):
        """BS7: qL = Z qG (masked entries of qL untouched)."""
        qL = torch.empty(self.NL, dtype=qG.dtype, device=qG.device) if qL is None else qL
        _check(getattr(lib(), "bs_scatter" + _sfx(qG))(self.handle, _ptr(qG, qG.dtype, "qG"),
                                                       _ptr(qL, qG.dtype, "qL"), _stream()),
               "bs_scatter")
        return qL

    def gather(self, qL, qG=None):
        """BS6: qG = Z^T qL."""
        qG = torch.empty(self.NG, dtype=qL.dtype, device=qL.device) if qG is None else qG
        _check(getattr(lib(), "bs_gather" + _sfx(qL))(self.handle, _ptr(qL, qL.dtype, "qL"),
                                                      _ptr(qG, qL.dtype, "qG"), _stream()),
               "bs_gather")
        return qG


class Rows:
    """A set of distinct rows of a map's Z^T in message order (bs_rows): the
    device steps of the multi-rank gather -- the continued row sums, and
    packing / unpacking row values into message buffers."""

    def __init__(self, m: Map, rows):
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        L = _bind(["bs_rows_create", "bs_rows_destroy", "bs_gather_rows", "bs_rows_pack",
                   "bs_rows_unpack"])
        h = ctypes.c_void_p()
        _check(L.bs_rows_create(m.handle, rows.size, rows.ctypes.data_as(ctypes.c_void_p),
                                ctypes.byref(h)), "bs_rows_create")
        self.handle, self.map, self.n = h, m, int(rows.size)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bs_rows_destroy(self.handle)
            self.handle = None

    def gather(self, qL, qG, start=None):
        """qG[rows[i]] = start[i] (or +0) + the row's copies in ascending order."""
        _check(lib().bs_gather_rows(self.handle, _ptr(qL, name="qL"), _ptr(start, name="start"),
                                    _ptr(qG, name="qG"), _stream()), "bs_gather_rows")
        return qG

    def pack(self, qG, out=None):
        """out[i] = qG[rows[i]]."""
        out = torch.empty(self.n, dtype=torch.float64, device=qG.device) if out is None else out
        _check(lib().bs_rows_pack(self.handle, _ptr(qG, name="qG"), _ptr(out, name="buf"),
                                  _stream()), "bs_rows_pack")
        return out

    def unpack(self, buf, qG):
        """qG[rows[i]] = buf[i]."""
        _check(lib().bs_rows_unpack(self.handle, _ptr(buf, name="buf"), _ptr(qG, name="qG"),
                                    _stream()), "bs_rows_unpack")
        return qG


# ---------------------------------------------------------------- operator and CG

class Problem:
    """A = Z^T (c S_L + lambda M_L) Z on a map (bs_problem); verts (host
    float64 [E, 8, 3], element corners) selects general hexahedra
    (bs_problem_create_geo; h is then unused)."""

    def __init__(self, m: Map, h: float, lam: float, coef=None, verts=None):
        self.map = m  # keep the map alive
        self.h, self.lam = h, lam
        c = None
        if coef is not None:
            self._coef = np.ascontiguousarray(coef, dtype=np.float64)
            c = self._coef.ctypes.data_as(ctypes.c_void_p)
        hd = ctypes.c_void_p()
        if verts is None:
            _check(lib().bs_problem_create(m.handle, h, lam, c, ctypes.byref(hd)),
                   "bs_problem_create")
        else:
            v = np.ascontiguousarray(verts, dtype=np.float64)
            _check(lib().bs_problem_create_geo(m.handle, lam, c, v.ctypes.data_as(ctypes.c_void_p),
                                               ctypes.byref(hd)), "bs_problem_create_geo")
        self.handle = hd

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bs_problem_destroy(self.handle)
            self.handle = None

    def apply_A(self, p, Ap=None):
        Ap = torch.empty_like(p) if Ap is None else Ap
        _check(lib().bs_apply_A(self.handle, _ptr(p), _ptr(Ap), _stream()), "bs_apply_A")
        return Ap

    def apply_A_ff(self, p, Ap=None):
        """A p with the float-float element operator (bs_apply_A_ff)."""
        Ap = torch.empty_like(p) if Ap is None else Ap
        _check(lib().bs_apply_A_ff(self.handle, _ptr(p), _ptr(Ap), _stream()), "bs_apply_A_ff")
        return Ap

    def apply_local(self, uL, AuL=None):
        AuL = torch.empty_like(uL) if AuL is None else AuL
        _check(lib().bs_apply_local(self.handle, _ptr(uL), _ptr(AuL), _stream()),
               "bs_apply_local")
        return AuL

    def diag(self, device=None):
        d = torch.empty(self.map.NG, dtype=torch.float64, device=device or "cuda")
        _check(lib().bs_diag_A(self.handle, _ptr(d), _stream()), "bs_diag_A")
        return d

    def cg(self, b, x=None, tol=1e-8, maxit=1000, flags=0, hist=None, check=True):
        """Algorithm 1.  Returns (x, info dict); hist (device, 3*(maxit+1))
        receives alpha_j, beta_j, rr_{j+1}."""
        if x is None:
            x = torch.zeros_like(b)
        info = CgInfo()
        rc = lib().bs_cg_solve(self.handle, _ptr(b), _ptr(x), tol, maxit, flags,
                               _ptr(hist) if hist is not None else None, ctypes.byref(info),
                               _stream())
        if check and rc not in (BS_OK,):
            _check(rc, "bs_cg_solve")
        d = info.as_dict()
        d["rc"] = rc
        return x, d

    def cg_refined_f32(self, b, x=None, tol=1e-10, maxit=1000000, inner_tol=1e-4,
                       outer_maxit=50, flags=0, check=True):
        """FP32 CG inside FP64 iterative refinement.  Returns (x, info dict);
        info['rel_residual'] is the FP64 true relative residual."""
        if x is None:
            x = torch.zeros_like(b)
        info = CgInfo()
        rc = lib().bs_cg_solve_refined_f32(self.handle, _ptr(b), _ptr(x), tol, maxit, inner_tol,
                                           outer_maxit, flags, ctypes.byref(info), _stream())
        if check and rc != BS_OK:
            _check(rc, "bs_cg_solve_refined_f32")
        d = info.as_dict()
        d["rc"] = rc
        return x, d


class BatchedConfig(ctypes.Structure):
    """bs_batched_config: chunk, blocks_per_sm, unroll (0 = default)."""
    _fields_ = [("chunk", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("unroll", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_SIGS.update({
    "bs_cg_solve_batched_ex": (ctypes.c_int, [_i32, _vp, _vp, _vp, _d, _i32, _i32,
                                              ctypes.POINTER(BatchedConfig),
                                              ctypes.POINTER(CgInfo), _vp]),
    "bs_cg_batched_autotune": (ctypes.c_int, [_i32, _vp, _vp, _i32, _i32,
                                              ctypes.POINTER(BatchedConfig),
                                              ctypes.POINTER(_d), _vp]),
})


def _arrays(problems, bs_, xs=None):
    n = len(problems)
    if n == 0 or n != len(bs_) or (xs is not None and n != len(xs)):
        raise ValueError("problems, b and x must be non-empty lists of one length")
    P = (ctypes.c_void_p * n)(*[p.handle.value for p in problems])
    B = (ctypes.c_void_p * n)(*[_ptr(b, name="b").value for b in bs_])
    X = None if xs is None else (ctypes.c_void_p * n)(*[_ptr(x, name="x").value for x in xs])
    return n, P, B, X


def solve_batched(problems, bs_, xs, tol=1e-8, maxit=1000000, flags=0, check=True, config=None):
    """bs_cg_solve_batched(_ex): Algorithm 1 on every (problem, b, x) together;
    config: a BatchedConfig or a dict of its fields (None: defaults).
    Returns (rc, list of per-solve info dicts)."""
    n, P, B, X = _arrays(problems, bs_, xs)
    infos = (CgInfo * n)()
    cfg = None
    if config is not None:
        cfg = config if isinstance(config, BatchedConfig) else BatchedConfig(**config)
    L = lib()
    if cfg is None:
        rc = L.bs_cg_solve_batched(n, ctypes.cast(P, ctypes.c_void_p),
                                   ctypes.cast(B, ctypes.c_void_p),
                                   ctypes.cast(X, ctypes.c_void_p), tol, maxit, flags, infos,
                                   _stream())
    else:
        _bind(["bs_cg_solve_batched_ex"])
        rc = L.bs_cg_solve_batched_ex(n, ctypes.cast(P, ctypes.c_void_p),
                                      ctypes.cast(B, ctypes.c_void_p),
                                      ctypes.cast(X, ctypes.c_void_p), tol, maxit, flags,
                                      ctypes.byref(cfg), infos, _stream())
    if check and rc != BS_OK:
        _check(rc, "bs_cg_solve_batched")
    return rc, [infos[i].as_dict() for i in range(n)]


def set_wait_budget(cycles=0):
    """bs_set_wait_budget: the batched solver's grid-barrier wait limit in SM
    clock cycles on the current device (cycles <= 0: the default).  Returns
    the previous limit."""
    L = _bind(["bs_set_wait_budget"])
    prev = ctypes.c_int64(0)
    _check(L.bs_set_wait_budget(int(cycles), ctypes.byref(prev)), "bs_set_wait_budget")
    return prev.value


def autotune_batched(problems, bs_, flags=0, iters=4):
    """bs_cg_batched_autotune: returns (BatchedConfig, ms per iteration)."""
    n, P, B, _ = _arrays(problems, bs_)
    L = _bind(["bs_cg_batched_autotune"])
    best = BatchedConfig()
    ms = ctypes.c_double(0.0)
    _check(L.bs_cg_batched_autotune(n, ctypes.cast(P, ctypes.c_void_p),
                                    ctypes.cast(B, ctypes.c_void_p), flags, iters,
                                    ctypes.byref(best), ctypes.byref(ms), _stream()),
           "bs_cg_batched_autotune")
    return best, ms.value


# ---------------------------------------------------------------- learned preconditioner

_SIGS.update({
    "bs_rows_create": (ctypes.c_int, [_vp, _i64, _vp, _pp]),
    "bs_rows_destroy": (ctypes.c_int, [_vp]),
    "bs_gather_rows": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "bs_rows_pack": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bs_rows_unpack": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bs_set_wait_budget": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "bs_gemm_engine": (ctypes.c_int, [_i32]),
    "bs_mlp_state_bytes": (ctypes.c_int64, [_vp]),
    "bs_mlp_save_state": (ctypes.c_int, [_vp, _vp, _i64]),
    "bs_mlp_load_state": (ctypes.c_int, [_vp, _vp, _i64]),
    "bs_mlp_create": (ctypes.c_int, [_i32, _i32, _vp, _vp, _i32, _pp]),
    "bs_mlp_destroy": (ctypes.c_int, [_vp]),
    "bs_mlp_get_weights": (ctypes.c_int, [_vp, _vp, _vp]),
    "bs_mlp_forward": (ctypes.c_int, [_vp, _i64, _vp, _vp, _i32, _vp]),
    "bs_mlp_loss_grad": (ctypes.c_int, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "bs_mlp_train_step": (ctypes.c_int, [_vp, _i64, _vp, _vp, _f, _vp, _vp]),
    "bs_mlp_pairs": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i32, _vp, _vp, _vp]),
    "bs_fpcg_learned": (ctypes.c_int, [_vp, _vp, _vp, _vp, _d, _i32, _i32,
                                       ctypes.POINTER(CgInfo), _vp]),
})


def _bind(names):
    L = lib()
    for n in names:
        res, args = _SIGS[n]
        f = getattr(L, n)
        f.restype, f.argtypes = res, args
    return L


def _fptr(t, name="tensor"):
    return _ptr(t, torch.float32, name)


def gemm_engine(engine=-1):
    """bs_gemm_engine: 0 mma.sync (default), 1 tcgen05; returns the previous
    engine (-1: query only)."""
    return _bind(["bs_gemm_engine"]).bs_gemm_engine(int(engine))


class MLP:
    """The element network y = W2 relu(W1 x) (bs_mlp): W1 [H x D], W2 [D x H]
    given as host float32 arrays (the caller draws the initial weights).
    split: BF16x3 operands (hi + lo bf16, three products) instead of BF16."""

    def __init__(self, W1, W2, split=False):
        W1 = np.ascontiguousarray(W1, dtype=np.float32)
        W2 = np.ascontiguousarray(W2, dtype=np.float32)
        H, D = W1.shape
        if W2.shape != (D, H):
            raise ValueError("W2 must be D x H")
        L = _bind(["bs_mlp_create", "bs_mlp_destroy", "bs_mlp_get_weights", "bs_mlp_forward",
                   "bs_mlp_loss_grad", "bs_mlp_train_step", "bs_mlp_pairs", "bs_fpcg_learned"])
        h = ctypes.c_void_p()
        _check(L.bs_mlp_create(D, H, W1.ctypes.data_as(ctypes.c_void_p),
                               W2.ctypes.data_as(ctypes.c_void_p),
                               BS_MLP_BF16X3 if split else 0, ctypes.byref(h)),
               "bs_mlp_create")
        self.handle, self.D, self.H, self.split = h, D, H, bool(split)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bs_mlp_destroy(self.handle)
            self.handle = None

    def weights(self):
        W1 = np.empty((self.H, self.D), np.float32)
        W2 = np.empty((self.D, self.H), np.float32)
        _check(lib().bs_mlp_get_weights(self.handle, W1.ctypes.data_as(ctypes.c_void_p),
                                        W2.ctypes.data_as(ctypes.c_void_p)), "bs_mlp_get_weights")
        return W1, W2

    def forward(self, X, odd=False):
        """f(X) row by row, or its odd part W2 W1 x / 2."""
        Y = torch.empty_like(X)
        _check(lib().bs_mlp_forward(self.handle, X.shape[0], _fptr(X, "X"), _fptr(Y, "Y"),
                                    BS_MLP_ODD if odd else 0, _stream()), "bs_mlp_forward")
        return Y

    def loss_grad(self, X, T):
        loss = torch.zeros(1, dtype=torch.float64, device=X.device)
        g1 = torch.empty((self.H, self.D), dtype=torch.float32, device=X.device)
        g2 = torch.empty((self.D, self.H), dtype=torch.float32, device=X.device)
        _check(lib().bs_mlp_loss_grad(self.handle, X.shape[0], _fptr(X, "X"), _fptr(T, "T"),
                                      _ptr(loss), _fptr(g1), _fptr(g2), _stream()),
               "bs_mlp_loss_grad")
        return loss, g1, g2

    def train_step(self, X, T, lr, loss=None):
        loss = torch.zeros(1, dtype=torch.float64, device=X.device) if loss is None else loss
        _check(lib().bs_mlp_train_step(self.handle, X.shape[0], _fptr(X, "X"), _fptr(T, "T"),
                                       float(lr), _ptr(loss), _stream()), "bs_mlp_train_step")
        return loss

    def save_state(self) -> bytes:
        """The training state (masters, Adam moments, step) as a host image
        (bs_mlp_save_state)."""
        L = _bind(["bs_mlp_state_bytes", "bs_mlp_save_state"])
        n = L.bs_mlp_state_bytes(self.handle)
        buf = ctypes.create_string_buffer(n)
        _check(L.bs_mlp_save_state(self.handle, buf, n), "bs_mlp_save_state")
        return buf.raw

    def load_state(self, image: bytes):
        """Restore a training state saved from a network of the same shape
        and mode (bs_mlp_load_state)."""
        L = _bind(["bs_mlp_load_state"])
        buf = ctypes.create_string_buffer(bytes(image), len(image))
        _check(L.bs_mlp_load_state(self.handle, buf, len(image)), "bs_mlp_load_state")

    def save(self, path):
        with open(path, "wb") as f:
            f.write(self.save_state())

    def load(self, path):
        with open(path, "rb") as f:
            self.load_state(f.read())


def mlp_pairs(problem, r, elems, negate_odd=False, out=None):
    """Training pairs (X, T) of the elements `elems` (int32 CUDA tensor) from a
    residual r (CUDA float64 N_G vector): X = u / rms, T = (e_I - u_I) / rms
    with e_I the element-interior error (bs_mlp_pairs)."""
    L = _bind(["bs_mlp_pairs"])
    Np = (problem.map.N + 1) ** 3
    n = elems.numel()
    if out is None:
        X = torch.empty((n, Np), dtype=torch.float32, device=r.device)
        T = torch.empty((n, Np), dtype=torch.float32, device=r.device)
    else:
        X, T = out
    _check(L.bs_mlp_pairs(problem.handle, _ptr(r), n, _ptr(elems, torch.int32),
                          int(bool(negate_odd)), _fptr(X), _fptr(T), _stream()), "bs_mlp_pairs")
    return X, T


def fpcg_learned(problem, mlp, b, x=None, tol=1e-8, maxit=100000, flags=0, check=True):
    """Flexible PCG with the learned correction (mlp None: Jacobi only).
    Returns (x, info dict)."""
    L = _bind(["bs_fpcg_learned"])
    x = torch.zeros_like(b) if x is None else x
    info = CgInfo()
    rc = L.bs_fpcg_learned(problem.handle, mlp.handle if mlp is not None else None, _ptr(b),
                           _ptr(x), tol, maxit, flags, ctypes.byref(info), _stream())
    if check and rc != BS_OK:
        _check(rc, "bs_fpcg_learned")
    d = info.as_dict()
    d["rc"] = rc
    return x, d
