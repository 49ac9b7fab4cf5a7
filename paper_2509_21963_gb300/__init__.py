"""GB300 (sm_103a) IterativeCUR: thin Python binding of the C ABI in include/cur.h.

The functions below carry the C names and only marshal arguments (ctypes);
every step of the method runs in the CUDA kernels of ``libcur.so``.  There is
no CPU fallback: if the library is missing the first call raises.

Typical use::

    import torch, paper_2509_21963_gb300 as cur
    ctx = cur.Context()                       # current device and torch stream
    res = ctx.run(A, tol=1e-6, block_size=10)  # A: CUDA float64/float32 matrix
    res.I, res.J, res.U, res.rho
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcur.so")

CUR_OK, CUR_EINVAL, CUR_ENONFINITE, CUR_ENOMEM, CUR_EBUDGET, CUR_ECUDA, CUR_ETIMEOUT, \
    CUR_TOL_UNREACHED = range(8)
CUR_F64, CUR_F32 = 0, 1
CUR_SKETCH_F64, CUR_SKETCH_BF16, CUR_SKETCH_BF16X2, CUR_SKETCH_BF16X3 = 0, 1, 2, 3
PHASES = ("gaussian", "sketch", "lupp_col", "row_res", "lupp_row", "factors", "col_res", "core")

_STATUS_NAMES = {0: "CUR_OK", 1: "CUR_EINVAL", 2: "CUR_ENONFINITE", 3: "CUR_ENOMEM",
                 4: "CUR_EBUDGET", 5: "CUR_ECUDA", 6: "CUR_ETIMEOUT", 7: "CUR_TOL_UNREACHED"}


class CurError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class cur_opts(ctypes.Structure):
    _fields_ = [("max_rank", ctypes.c_int64), ("omega", ctypes.c_void_p),
                ("sketch_mode", ctypes.c_int), ("alpha", ctypes.c_double),
                ("delta", ctypes.c_double), ("timing", ctypes.c_int)]


_lib = None
_vp, _i64, _dbl, _u64, _int, _sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                    ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t)

_SIGNATURES = {
    "cur_create": (_int, [ctypes.POINTER(_vp), _int, _vp, _sz]),
    "cur_free": (None, [_vp]),
    "cur_last_error": (ctypes.c_char_p, [_vp]),
    "cur_run": (_int, [_vp, _vp, _i64, _i64, _i64, _int, _dbl, _int, _int, _u64,
                       ctypes.POINTER(_vp)]),
    "cur_run_opts": (_int, [_vp, _vp, _i64, _i64, _i64, _int, _dbl, _int, _int, _u64,
                            ctypes.POINTER(cur_opts), ctypes.POINTER(_vp)]),
    "cur_run_host": (_int, [_vp, _vp, _i64, _i64, _i64, _int, _dbl, _int, _int, _u64,
                            ctypes.POINTER(cur_opts), ctypes.POINTER(_vp)]),
    "cur_result_rank": (_i64, [_vp]),
    "cur_result_iterations": (_i64, [_vp]),
    "cur_result_status": (_int, [_vp]),
    "cur_result_err": (_dbl, [_vp]),
    "cur_result_sketch_norm": (_dbl, [_vp]),
    "cur_result_I": (_vp, [_vp]),
    "cur_result_J": (_vp, [_vp]),
    "cur_result_U": (_vp, [_vp]),
    "cur_result_rho_history": (ctypes.POINTER(_dbl), [_vp]),
    "cur_result_phase_ms": (_dbl, [_vp, _int]),
    "cur_result_kernel_launches": (_i64, [_vp]),
    "cur_result_copy_to_host": (_int, [_vp, _vp, _vp, _vp]),
    "cur_result_free": (None, [_vp]),
    "cur_step_gaussian": (_int, [_vp, _u64, _i64, _i64, _vp]),
    "cur_step_sketch": (_int, [_vp, _vp, _i64, _vp, _i64, _i64, _i64, _int, _vp, _vp]),
    "cur_step_sketch_q": (_int, [_vp, _vp, _i64, _vp, _i64, _i64, _i64, _int, _vp, _vp]),
    "cur_step_lupp": (_int, [_vp, _vp, _i64, _i64, _i64, _i64, _vp, _vp]),
    "cur_step_pinv": (_int, [_vp, _vp, _i64, _i64, _i64, _dbl, _vp, _vp]),
    "cur_step_lupp_noalloc": (_int, [_int, _vp, _vp, _i64, _i64, _i64, _i64, _vp, _vp,
                                     ctypes.c_char_p, _sz]),
}

EXPORTED = tuple(_SIGNATURES)


def lib():
    """Load libcur.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; run "
                               "python -c 'import __graft_entry__ as g; g.build()'")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def __getattr__(name):  # cur_* names resolve to the C functions
    if name in _SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


def _check(ctx_ptr, status, ok=(CUR_OK,)):
    if status not in ok:
        msg = lib().cur_last_error(ctx_ptr) or b""
        raise CurError(status, msg.decode())
    return status


@dataclass
class Result:
    rank: int
    iterations: int
    status: int
    rho: float
    sketch_norm: float
    rho_history: np.ndarray
    kernel_launches: int
    phase_ms: dict
    I: np.ndarray = field(repr=False)
    J: np.ndarray = field(repr=False)
    U: np.ndarray = field(repr=False)


def _result_from(ptr) -> Result:
    L = lib()
    r = int(L.cur_result_rank(ptr))
    k = int(L.cur_result_iterations(ptr))
    hist = L.cur_result_rho_history(ptr)
    rh = np.array([hist[i] for i in range(k)], dtype=np.float64) if k else np.zeros(0)
    I = np.zeros(r, dtype=np.int64)
    J = np.zeros(r, dtype=np.int64)
    U = np.zeros((r, r), dtype=np.float64)
    if r:
        st = L.cur_result_copy_to_host(ptr, I.ctypes.data, J.ctypes.data, U.ctypes.data)
        if st != CUR_OK:
            raise CurError(st, "copy to host failed")
    return Result(rank=r, iterations=k, status=int(L.cur_result_status(ptr)),
                  rho=float(L.cur_result_err(ptr)), sketch_norm=float(L.cur_result_sketch_norm(ptr)),
                  rho_history=rh, kernel_launches=int(L.cur_result_kernel_launches(ptr)),
                  phase_ms={p: float(L.cur_result_phase_ms(ptr, i)) for i, p in enumerate(PHASES)},
                  I=I, J=J, U=U)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return CUR_F64
    if t.dtype == torch.float32:
        return CUR_F32
    raise TypeError(f"A must be float64 or float32, got {t.dtype}")


class Context:
    """Owns a cur_ctx bound to one device and one CUDA stream."""

    def __init__(self, device: int | None = None, stream=None, hbm_budget_bytes: int = 0):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.device = device
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        self.ptr = _vp()
        _check(None, lib().cur_create(ctypes.byref(self.ptr), device, _vp(handle), hbm_budget_bytes))

    def close(self):
        if self.ptr:
            lib().cur_free(self.ptr)
            self.ptr = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return (lib().cur_last_error(self.ptr) or b"").decode()

    @staticmethod
    def _opts(max_rank=0, omega=None, alpha=0.0, delta=0.0, sketch_mode=CUR_SKETCH_F64, timing=False):
        o = cur_opts()
        o.timing = 1 if timing else 0
        o.max_rank = max_rank
        o.omega = omega.data_ptr() if omega is not None else None
        o.sketch_mode = sketch_mode
        o.alpha = alpha
        o.delta = delta
        return o

    def run_raw(self, A, tol, block_size, sketch_size=0, seed=0, **kw):
        """cur_run_opts on a CUDA tensor; returns (status, result pointer)."""
        assert A.is_cuda and A.dim() == 2 and A.stride(1) == 1
        m, n = A.shape
        out = _vp()
        o = self._opts(**kw)
        st = lib().cur_run_opts(self.ptr, _vp(A.data_ptr()), m, n, A.stride(0), _dtype_code(A),
                                float(tol), int(block_size), int(sketch_size), int(seed),
                                ctypes.byref(o), ctypes.byref(out))
        return st, out

    def run(self, A, tol, block_size, sketch_size=0, seed=0, **kw) -> Result:
        st, out = self.run_raw(A, tol, block_size, sketch_size, seed, **kw)
        _check(self.ptr, st, ok=(CUR_OK, CUR_TOL_UNREACHED))
        try:
            return _result_from(out)
        finally:
            lib().cur_result_free(out)

    def run_host(self, A: np.ndarray, tol, block_size, sketch_size=0, seed=0, **kw) -> Result:
        """End-to-end form: A is a host array (C-contiguous float64/float32)."""
        assert A.ndim == 2 and A.flags.c_contiguous
        dt = {np.dtype(np.float64): CUR_F64, np.dtype(np.float32): CUR_F32}[A.dtype]
        out = _vp()
        o = self._opts(**kw)
        st = lib().cur_run_host(self.ptr, _vp(A.ctypes.data), A.shape[0], A.shape[1], A.shape[1], dt,
                                float(tol), int(block_size), int(sketch_size), int(seed),
                                ctypes.byref(o), ctypes.byref(out))
        _check(self.ptr, st, ok=(CUR_OK, CUR_TOL_UNREACHED))
        try:
            return _result_from(out)
        finally:
            lib().cur_result_free(out)

    # ---- single steps (include/cur_steps.h) ----
    def gaussian(self, seed: int, c: int, m: int):
        import torch
        G = torch.empty(c, m, dtype=torch.float64, device=f"cuda:{self.device}")
        _check(self.ptr, lib().cur_step_gaussian(self.ptr, seed, c, m, _vp(G.data_ptr())))
        return G

    def sketch(self, G, A):
        import torch
        c, m = G.shape
        n = A.shape[1]
        Y = torch.empty(c, n, dtype=torch.float64, device=A.device)
        ss = ctypes.c_double()
        _check(self.ptr, lib().cur_step_sketch(self.ptr, _vp(G.data_ptr()), c, _vp(A.data_ptr()), m, n,
                                               A.stride(0), _dtype_code(A), _vp(Y.data_ptr()),
                                               ctypes.byref(ss)))
        return Y, ss.value

    def sketch_q(self, G, A, digits: int):
        """Precision-form sketch Y = G_q fix_S(A) (A: CUDA float32)."""
        import torch
        c, m = G.shape
        n = A.shape[1]
        Y = torch.empty(c, n, dtype=torch.float64, device=A.device)
        ss = ctypes.c_double()
        _check(self.ptr, lib().cur_step_sketch_q(self.ptr, _vp(G.data_ptr()), c, _vp(A.data_ptr()), m,
                                                 n, A.stride(0), int(digits), _vp(Y.data_ptr()),
                                                 ctypes.byref(ss)))
        return Y, ss.value

    def lupp(self, X, steps: int, mask=None):
        import torch
        nr, ncand = X.shape
        if mask is None:
            mask = torch.zeros(ncand, dtype=torch.uint8, device=X.device)
        piv = torch.full((steps,), -1, dtype=torch.int64, device=X.device)
        _check(self.ptr, lib().cur_step_lupp(self.ptr, _vp(X.data_ptr()), X.stride(0), nr, ncand, steps,
                                             _vp(mask.data_ptr()), _vp(piv.data_ptr())))
        return piv, mask

    def pinv(self, M, thr: float = -1.0):
        import torch
        p, q = M.shape
        X = torch.empty(q, p, dtype=torch.float64, device=M.device)
        k = ctypes.c_int64()
        _check(self.ptr, lib().cur_step_pinv(self.ptr, _vp(M.data_ptr()), p, q, M.stride(0), float(thr),
                                             _vp(X.data_ptr()), ctypes.byref(k)))
        return X, k.value
