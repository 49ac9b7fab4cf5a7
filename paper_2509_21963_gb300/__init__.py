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
CUR_SKETCH_F64, CUR_SKETCH_BF16, CUR_SKETCH_BF16X2, CUR_SKETCH_BF16X3, CUR_SKETCH_BF16X4 = 0, 1, 2, 3, 4
CUR_SKETCH_F64_TC = 5
PHASES = ("gaussian", "sketch", "lupp_col", "row_res", "lupp_row", "factors", "col_res", "core",
          "scales")

_STATUS_NAMES = {0: "CUR_OK", 1: "CUR_EINVAL", 2: "CUR_ENONFINITE", 3: "CUR_ENOMEM",
                 4: "CUR_EBUDGET", 5: "CUR_ECUDA", 6: "CUR_ETIMEOUT", 7: "CUR_TOL_UNREACHED"}


class CurError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class cur_opts(ctypes.Structure):
    _fields_ = [("max_rank", ctypes.c_int64), ("omega", ctypes.c_void_p),
                ("sketch_mode", ctypes.c_int), ("alpha", ctypes.c_double),
                ("delta", ctypes.c_double), ("timing", ctypes.c_int),
                ("residual_planes", ctypes.c_int)]


class cur_batch_job(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("tol", ctypes.c_double), ("block_size", ctypes.c_int32),
                ("sketch_size", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("max_rank", ctypes.c_int64)]


class cur_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("waves", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t),
                ("budget", ctypes.c_size_t), ("pending", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("launches", ctypes.c_int64)]


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
    "cur_step_sketch_fx": (_int, [_vp, _vp, _i64, _vp, _i64, _i64, _i64, _vp, _vp]),
    "cur_probe_fp64_tflops": (_int, [_vp, ctypes.POINTER(_dbl)]),
    "cur_probe_latency": (_int, [_vp, ctypes.POINTER(_dbl), _int]),
    "cur_test_wait_timeout": (_int, [_vp, _int, _int, _dbl]),
    "cur_step_lupp": (_int, [_vp, _vp, _i64, _i64, _i64, _i64, _vp, _vp]),
    "cur_step_pinv": (_int, [_vp, _vp, _i64, _i64, _i64, _dbl, _vp, _vp]),
    "cur_step_gemm": (_int, [_vp, _i64, _i64, _i64, _dbl, _vp, _i64, _int, _vp, _i64, _int, _dbl,
                             _vp, _i64, _vp, _i64, _vp]),
    "cur_step_resid_tc": (_int, [_vp, _vp, _i64, _vp, _i64, _i64, _i64, _i64, _int, _vp, _i64]),
    "cur_step_gather": (_int, [_vp, _vp, _i64, _int, _vp, _vp, _i64, _i64, _i64, _i64, _vp, _i64]),
    "cur_step_lupp_noalloc": (_int, [_int, _vp, _vp, _i64, _i64, _i64, _i64, _vp, _vp,
                                     ctypes.c_char_p, _sz]),
    "cur_batch_create": (_int, [_vp, ctypes.POINTER(cur_batch_job), _i64, _int, ctypes.POINTER(_vp)]),
    "cur_batch_free": (None, [_vp]),
    "cur_batch_set_team": (_int, [_vp, _int]),
    "cur_batch_set_classes": (_int, [_vp, _int, _int, _int, _i64]),
    "cur_batch_set_tile": (_int, [_vp, _int]),
    "cur_batch_get_tile": (_int, [_vp, ctypes.POINTER(_int)]),
    "cur_batch_get_classes": (_int, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int),
                                     ctypes.POINTER(_i64)]),
    "cur_batch_get_schedule": (_int, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int),
                                      ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "cur_batch_tune": (_int, [_vp, ctypes.POINTER(_int), _int, ctypes.POINTER(_int),
                              ctypes.POINTER(_dbl)]),
    "cur_batch_phase_cycles": (_int, [_vp, ctypes.POINTER(_dbl), _int]),
    "cur_batch_job_cycles": (_int, [_vp, _i64, ctypes.POINTER(_i64)]),
    "cur_batch_launch": (_int, [_vp]),
    "cur_batch_wait": (_int, [_vp]),
    "cur_batch_run": (_int, [_vp]),
    "cur_batch_job_result": (_int, [_vp, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                    ctypes.POINTER(_dbl), ctypes.POINTER(_int)]),
    "cur_batch_I": (_vp, [_vp, _i64]),
    "cur_batch_J": (_vp, [_vp, _i64]),
    "cur_batch_U": (_vp, [_vp, _i64]),
    "cur_batch_rho_history": (_vp, [_vp, _i64]),
    "cur_batch_copy_job": (_int, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "cur_server_create": (_int, [_vp, _sz, _int, _int, _int, _i64, _int, ctypes.POINTER(_vp)]),
    "cur_server_free": (None, [_vp]),
    "cur_server_submit": (_int, [_vp, ctypes.POINTER(cur_batch_job), _int, ctypes.POINTER(_u64)]),
    "cur_server_wait": (_int, [_vp, _u64, _dbl]),
    "cur_server_poll": (_int, [_vp, _u64, ctypes.POINTER(_int)]),
    "cur_server_drain": (_int, [_vp]),
    "cur_server_result": (_int, [_vp, _u64, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                 ctypes.POINTER(_dbl), ctypes.POINTER(_int), ctypes.POINTER(_dbl),
                                 ctypes.POINTER(_dbl)]),
    "cur_server_copy": (_int, [_vp, _u64, _vp, _vp, _vp, _vp]),
    "cur_server_release": (_int, [_vp, _u64]),
    "cur_server_get_stats": (_int, [_vp, ctypes.POINTER(cur_server_stats)]),
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
    def _opts(max_rank=0, omega=None, alpha=0.0, delta=0.0, sketch_mode=CUR_SKETCH_F64, timing=False,
              residual_planes=0):
        o = cur_opts()
        o.residual_planes = residual_planes
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
        """End-to-end form: A is a host array (float64/float32, rows contiguous,
        row stride a whole number of elements >= n)."""
        assert A.ndim == 2 and A.strides[1] == A.itemsize and A.strides[0] % A.itemsize == 0
        lda = A.strides[0] // A.itemsize
        assert lda >= A.shape[1]
        dt = {np.dtype(np.float64): CUR_F64, np.dtype(np.float32): CUR_F32}[A.dtype]
        out = _vp()
        o = self._opts(**kw)
        st = lib().cur_run_host(self.ptr, _vp(A.ctypes.data), A.shape[0], A.shape[1], lda, dt,
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

    def sketch_fx(self, G, A):
        """FP64 tensor-core sketch Y = RN(G_q trunc(A 2^(52-E))) 2^(E-52) (A: CUDA float64)."""
        import torch
        c, m = G.shape
        n = A.shape[1]
        Y = torch.empty(c, n, dtype=torch.float64, device=A.device)
        ss = ctypes.c_double()
        _check(self.ptr, lib().cur_step_sketch_fx(self.ptr, _vp(G.data_ptr()), c, _vp(A.data_ptr()), m,
                                                  n, A.stride(0), _vp(Y.data_ptr()), ctypes.byref(ss)))
        return Y, ss.value

    def wait_timeout_status(self, which: int, nblocks: int = 2, budget_ms: float = 2.0) -> int:
        """Status of cur_test_wait_timeout (CUR_ETIMEOUT when the bounded wait gave up)."""
        return lib().cur_test_wait_timeout(self.ptr, int(which), int(nblocks), float(budget_ms))

    LATENCY_KINDS = ("dfma", "dfma_one_lane", "dadd", "shfl_dadd", "ddiv", "dsqrt_add",
                     "dsetp_select", "ffma", "shfl_i64_max", "l2_load")

    def latency_cycles(self) -> dict:
        """Cycles per dependent operation (include/cur_steps.h, cur_probe_latency)."""
        arr = (_dbl * len(self.LATENCY_KINDS))()
        _check(self.ptr, lib().cur_probe_latency(self.ptr, arr, len(self.LATENCY_KINDS)))
        return dict(zip(self.LATENCY_KINDS, list(arr)))

    def fp64_tflops(self) -> float:
        """Measured FP64 FMA rate of the device (TFLOP/s)."""
        v = ctypes.c_double()
        _check(self.ptr, lib().cur_probe_fp64_tflops(self.ptr, ctypes.byref(v)))
        return v.value

    def lupp(self, X, steps: int, mask=None):
        import torch
        nr, ncand = X.shape
        if mask is None:
            mask = torch.zeros(ncand, dtype=torch.uint8, device=X.device)
        piv = torch.full((steps,), -1, dtype=torch.int64, device=X.device)
        _check(self.ptr, lib().cur_step_lupp(self.ptr, _vp(X.data_ptr()), X.stride(0), nr, ncand, steps,
                                             _vp(mask.data_ptr()), _vp(piv.data_ptr())))
        return piv, mask

    def gemm(self, alpha, A, B, beta=0.0, C=None, out=None, trans_a=False, trans_b=False,
             sumsq=False):
        """D = alpha op(A) op(B) + beta C (FP64 CUDA tensors, unit column
        stride); `out` may be C.  Returns D, or (D, ||D||_F^2) with sumsq."""
        import torch
        M = A.shape[1] if trans_a else A.shape[0]
        K = A.shape[0] if trans_a else A.shape[1]
        N = B.shape[0] if trans_b else B.shape[1]
        if out is None:
            out = torch.empty(M, N, dtype=torch.float64, device=A.device)
        ss = ctypes.c_double()
        cptr = C.data_ptr() if (C is not None and beta != 0.0) else None
        ldc = C.stride(0) if (C is not None and beta != 0.0) else 0
        _check(self.ptr, lib().cur_step_gemm(self.ptr, M, N, K, float(alpha), _vp(A.data_ptr()),
                                             A.stride(0), int(trans_a), _vp(B.data_ptr()),
                                             B.stride(0), int(trans_b), float(beta), _vp(cptr),
                                             ldc, _vp(out.data_ptr()), out.stride(0),
                                             ctypes.byref(ss) if sumsq else None))
        return (out, ss.value) if sumsq else out

    def resid_tc(self, P, Q, D, planes: int = 2):
        """D(n, i) -= sum_k P(i, k) Q(n, k) on the tensor cores (FP64 CUDA tensors;
        P: M x K, Q: N x K, D: N x M), in place; returns D."""
        M, K = P.shape
        N = Q.shape[0]
        _check(self.ptr, lib().cur_step_resid_tc(self.ptr, _vp(P.data_ptr()), P.stride(0),
                                                 _vp(Q.data_ptr()), Q.stride(0), M, N, K, int(planes),
                                                 _vp(D.data_ptr()), D.stride(0)))
        return D

    def gather(self, X, rows, cols, ridx=None, cidx=None, trans=False, out=None):
        """out[a, t] = X(ridx[a], cidx[t]) (X^T's entries when trans); indices
        outside X give 0.0.  ridx / cidx: int64 CUDA tensors or None."""
        import torch
        if out is None:
            out = torch.empty(rows, cols, dtype=torch.float64, device=X.device)
        rlim, clim = (X.shape[1], X.shape[0]) if trans else (X.shape[0], X.shape[1])
        _check(self.ptr, lib().cur_step_gather(
            self.ptr, _vp(X.data_ptr()), X.stride(0), int(trans),
            _vp(ridx.data_ptr() if ridx is not None else None),
            _vp(cidx.data_ptr() if cidx is not None else None),
            rows, cols, rlim, clim, _vp(out.data_ptr()), out.stride(0)))
        return out

    def pinv(self, M, thr: float = -1.0):
        import torch
        p, q = M.shape
        X = torch.empty(q, p, dtype=torch.float64, device=M.device)
        k = ctypes.c_int64()
        _check(self.ptr, lib().cur_step_pinv(self.ptr, _vp(M.data_ptr()), p, q, M.stride(0), float(thr),
                                             _vp(X.data_ptr()), ctypes.byref(k)))
        return X, k.value


@dataclass
class BatchJobResult:
    rank: int
    iterations: int
    status: int
    rho: float
    rho_history: np.ndarray = field(repr=False)
    I: np.ndarray = field(repr=False)
    J: np.ndarray = field(repr=False)
    U: np.ndarray = field(repr=False)


class Batch:
    """Many independent decompositions in one persistent launch
    (include/cur_batch.h).  `mats` is a list of CUDA tensors of one dtype
    (row stride >= columns, unit column stride); tol, block_size, sketch_size,
    seed and max_rank are scalars or per-job sequences.  The tensors are
    borrowed: they must stay alive and unchanged while the batch exists."""

    def __init__(self, ctx: Context, mats, tol, block_size, sketch_size=0, seed=0, max_rank=0):
        k = len(mats)
        per = lambda v: list(v) if isinstance(v, (list, tuple, np.ndarray)) else [v] * k  # noqa: E731
        tols, bs, cs, seeds, mrs = per(tol), per(block_size), per(sketch_size), per(seed), per(max_rank)
        self.ctx = ctx
        self.mats = list(mats)
        jobs = (cur_batch_job * k)()
        dt = _dtype_code(self.mats[0])
        for j, A in enumerate(self.mats):
            if not (A.is_cuda and A.dim() == 2 and A.stride(1) == 1):
                raise ValueError(f"job {j}: A must be a 2-D CUDA tensor with unit column stride")
            if _dtype_code(A) != dt:
                raise TypeError(f"job {j}: every matrix of a batch has the dtype of the first")
            jobs[j].A = A.data_ptr()
            jobs[j].m, jobs[j].n = A.shape
            jobs[j].lda = A.stride(0)
            jobs[j].tol = float(tols[j])
            jobs[j].block_size = int(bs[j])
            jobs[j].sketch_size = int(cs[j])
            jobs[j].seed = int(seeds[j])
            jobs[j].max_rank = int(mrs[j])
        self.njobs = k
        self.ptr = _vp()
        _check(ctx.ptr, lib().cur_batch_create(ctx.ptr, jobs, k, dt, ctypes.byref(self.ptr)))

    def close(self):
        if getattr(self, "ptr", None):
            lib().cur_batch_free(self.ptr)
            self.ptr = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self):
        _check(self.ctx.ptr, lib().cur_batch_run(self.ptr))

    def launch(self):
        _check(self.ctx.ptr, lib().cur_batch_launch(self.ptr))

    def wait(self):
        _check(self.ctx.ptr, lib().cur_batch_wait(self.ptr))

    def set_team(self, team: int):
        _check(self.ctx.ptr, lib().cur_batch_set_team(self.ptr, int(team)))

    def set_classes(self, team: int, team_big: int, nbig: int, big_cut: int):
        """nbig teams of team_big CTAs take the big_cut largest jobs first; the
        other CTAs form teams of `team` (include/cur_batch.h)."""
        _check(self.ctx.ptr, lib().cur_batch_set_classes(self.ptr, int(team), int(team_big),
                                                         int(nbig), int(big_cut)))

    def set_tile(self, tile_n: int):
        _check(self.ctx.ptr, lib().cur_batch_set_tile(self.ptr, int(tile_n)))

    def tune(self, candidates=None):
        best, ms = _int(), _dbl()
        if candidates is None:
            _check(self.ctx.ptr, lib().cur_batch_tune(self.ptr, None, 0, ctypes.byref(best),
                                                      ctypes.byref(ms)))
        else:
            arr = (_int * len(candidates))(*candidates)
            _check(self.ctx.ptr, lib().cur_batch_tune(self.ptr, arr, len(candidates),
                                                      ctypes.byref(best), ctypes.byref(ms)))
        return best.value, ms.value

    def schedule(self) -> dict:
        t, g, n, gr = _int(), _int(), _int(), _int()
        _check(self.ctx.ptr, lib().cur_batch_get_schedule(self.ptr, ctypes.byref(t), ctypes.byref(g),
                                                          ctypes.byref(n), ctypes.byref(gr)))
        tb, nb, cut = _int(), _int(), _i64()
        _check(self.ctx.ptr, lib().cur_batch_get_classes(self.ptr, ctypes.byref(tb), ctypes.byref(nb),
                                                         ctypes.byref(cut)))
        tile = _int()
        _check(self.ctx.ptr, lib().cur_batch_get_tile(self.ptr, ctypes.byref(tile)))
        return {"team": t.value, "grid": g.value, "teams": n.value, "graph": bool(gr.value),
                "team_big": tb.value, "nbig": nb.value, "big_cut": cut.value, "tile_n": tile.value}

    BATCH_PHASES = ("sketch", "lupp_col", "row_res", "lupp_row", "updates", "core_factor",
                    "core_solve", "jobs")

    def phase_cycles(self) -> dict:
        v = (_dbl * 8)()
        _check(self.ctx.ptr, lib().cur_batch_phase_cycles(self.ptr, v, 8))
        return {k: v[i] for i, k in enumerate(self.BATCH_PHASES)}

    def job_cycles(self, j: int) -> int:
        v = _i64()
        _check(self.ctx.ptr, lib().cur_batch_job_cycles(self.ptr, j, ctypes.byref(v)))
        return int(v.value)

    def info(self, j: int):
        r, it, rho, st = _i64(), _i64(), _dbl(), _int()
        _check(self.ctx.ptr, lib().cur_batch_job_result(self.ptr, j, ctypes.byref(r), ctypes.byref(it),
                                                        ctypes.byref(rho), ctypes.byref(st)))
        return int(r.value), int(it.value), float(rho.value), int(st.value)

    def result(self, j: int) -> BatchJobResult:
        r, it, rho, st = self.info(j)
        I = np.zeros(r, dtype=np.int64)
        J = np.zeros(r, dtype=np.int64)
        U = np.zeros((r, r), dtype=np.float64)
        h = np.zeros(it, dtype=np.float64)
        _check(self.ctx.ptr, lib().cur_batch_copy_job(self.ptr, j, I.ctypes.data, J.ctypes.data,
                                                      U.ctypes.data, h.ctypes.data))
        return BatchJobResult(rank=r, iterations=it, status=st, rho=rho, rho_history=h, I=I, J=J, U=U)


@dataclass
class ServedResult:
    rank: int
    iterations: int
    status: int
    rho: float
    latency_ms: float
    queue_ms: float
    rho_history: np.ndarray = field(repr=False)
    I: np.ndarray = field(repr=False)
    J: np.ndarray = field(repr=False)
    U: np.ndarray = field(repr=False)
    error: str = ""  # why the request failed (status other than OK / TOL_UNREACHED)


class Server:
    """Serving form (include/cur_server.h): submit requests, the scheduler
    thread admits them by HBM footprint and runs them in overlapping waves."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, dtype="float32", team: int = 4,
                 streams: int = 4, big_elements: int = 0, big_lanes: int = 1):
        self.ctx = ctx
        self.dtype = CUR_F32 if str(dtype).endswith("32") else CUR_F64
        self._keep = {}
        self.ptr = _vp()
        _check(ctx.ptr, lib().cur_server_create(ctx.ptr, int(hbm_budget_bytes), self.dtype, int(team),
                                                int(streams), int(big_elements), int(big_lanes),
                                                ctypes.byref(self.ptr)))

    def close(self):
        if getattr(self, "ptr", None):
            lib().cur_server_free(self.ptr)
            self.ptr = _vp()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, A, tol, block_size, sketch_size=0, seed=0, max_rank=0) -> int:
        """A: a CUDA tensor (borrowed until the request completes) or a
        C-contiguous numpy array (host request, copied at admission)."""
        j = cur_batch_job()
        on_host = isinstance(A, np.ndarray)
        if on_host:
            if not A.flags.c_contiguous:
                raise ValueError("host A must be C-contiguous")
            want = np.float32 if self.dtype == CUR_F32 else np.float64
            if A.dtype != want:
                raise TypeError(f"server dtype is {np.dtype(want).name}")
            j.A = A.ctypes.data
            j.m, j.n = A.shape
            j.lda = A.shape[1]
        else:
            if not (A.is_cuda and A.dim() == 2 and A.stride(1) == 1):
                raise ValueError("A must be a 2-D CUDA tensor with unit column stride")
            if _dtype_code(A) != self.dtype:
                raise TypeError("A's dtype differs from the server's")
            j.A = A.data_ptr()
            j.m, j.n = A.shape
            j.lda = A.stride(0)
        j.tol = float(tol)
        j.block_size = int(block_size)
        j.sketch_size = int(sketch_size)
        j.seed = int(seed)
        j.max_rank = int(max_rank)
        t = _u64()
        _check(self.ctx.ptr, lib().cur_server_submit(self.ptr, ctypes.byref(j), 1 if on_host else 0,
                                                     ctypes.byref(t)))
        self._keep[t.value] = A
        return t.value

    def wait(self, ticket: int, timeout_s: float = -1.0):
        _check(self.ctx.ptr, lib().cur_server_wait(self.ptr, ticket, float(timeout_s)))

    def poll(self, ticket: int) -> bool:
        d = _int()
        _check(self.ctx.ptr, lib().cur_server_poll(self.ptr, ticket, ctypes.byref(d)))
        return bool(d.value)

    def drain(self):
        _check(self.ctx.ptr, lib().cur_server_drain(self.ptr))

    def info(self, ticket: int):
        r, it, rho, st, lat, q = _i64(), _i64(), _dbl(), _int(), _dbl(), _dbl()
        _check(self.ctx.ptr, lib().cur_server_result(self.ptr, ticket, ctypes.byref(r), ctypes.byref(it),
                                                     ctypes.byref(rho), ctypes.byref(st),
                                                     ctypes.byref(lat), ctypes.byref(q)))
        return int(r.value), int(it.value), float(rho.value), int(st.value), lat.value, q.value

    def result(self, ticket: int, release: bool = True) -> ServedResult:
        r, it, rho, st, lat, q = self.info(ticket)
        err = "" if st in (CUR_OK, CUR_TOL_UNREACHED) else self.ctx.last_error()
        I = np.zeros(r, dtype=np.int64)
        J = np.zeros(r, dtype=np.int64)
        U = np.zeros((r, r), dtype=np.float64)
        h = np.zeros(it, dtype=np.float64)
        _check(self.ctx.ptr, lib().cur_server_copy(self.ptr, ticket, I.ctypes.data, J.ctypes.data,
                                                   U.ctypes.data, h.ctypes.data))
        if release:
            self.release(ticket)
        return ServedResult(rank=r, iterations=it, status=st, rho=rho, latency_ms=lat, queue_ms=q,
                            rho_history=h, I=I, J=J, U=U, error=err)

    def release(self, ticket: int):
        _check(self.ctx.ptr, lib().cur_server_release(self.ptr, ticket))
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        o = cur_server_stats()
        _check(self.ctx.ptr, lib().cur_server_get_stats(self.ptr, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in cur_server_stats._fields_}
