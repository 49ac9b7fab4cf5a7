"""FP64 CPU oracle of IterativeCUR (arXiv 2509.21963, Algorithm 1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library under ``paper_2509_21963_gb300/``: the arithmetic lives in
``cur_oracle.c`` (plain C, compiled with ``-ffp-contract=off``); this module only
compiles it and marshals numpy arrays through ctypes.

Parity status: each function is pinned by ``tests/test_oracle_pins.py`` or
``tests/test_oracle_precision_pins.py``; the header of ``cur_oracle.c`` lists
which pin covers which function.  The precision-form functions (the 8-bit
sketch, the fixed points, the exact fixed-point sketch) are this project's own
definitions, pinned to the error bounds and exact rational values they state.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cur_oracle.c")
_HDR = os.path.join(_HERE, "cur_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libcur_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile cur_oracle.c into oracle/_build/libcur_oracle.so (gcc, -O2)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(f) > os.path.getmtime(_LIB) for f in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                "-o", tmp, _SRC, "-lm"]
        # OpenMP over independent outer loops only (no split reductions), so the
        # arithmetic is that of the serial build; without libgomp, build serial
        r = subprocess.run(base[:-1] + ["-fopenmp", "-lm"], capture_output=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Out(ctypes.Structure):
    _fields_ = [
        ("I", ctypes.c_void_p), ("J", ctypes.c_void_p), ("U", ctypes.c_void_p),
        ("rho_hist", ctypes.c_void_p), ("gap_col", ctypes.c_void_p),
        ("gap_row", ctypes.c_void_p), ("scale_row", ctypes.c_void_p),
        ("S_final", ctypes.c_void_p), ("hist_cap", ctypes.c_int64),
        ("rank", ctypes.c_int64), ("iters", ctypes.c_int64),
        ("rho", ctypes.c_double), ("normY", ctypes.c_double),
        ("maxabsY", ctypes.c_double), ("status", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        vp, i64, dbl, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        L.cur_oracle_philox4x64_10.argtypes = [vp, vp, vp]
        L.cur_oracle_gaussian_sketch.argtypes = [u64, i64, i64, vp]
        L.cur_oracle_sketch.argtypes = [vp, i64, vp, i64, i64, i64, vp]
        L.cur_oracle_lupp.argtypes = [vp, i64, i64, i64, i64, vp, vp, vp]
        L.cur_oracle_lupp.restype = ctypes.c_int
        L.cur_oracle_qrcp_pinv.argtypes = [vp, i64, i64, i64, dbl, vp, vp, vp]
        L.cur_oracle_qrcp_pinv.restype = i64
        L.cur_oracle_run.argtypes = [vp, i64, i64, i64, dbl, i64, i64, u64, vp, i64,
                                     ctypes.c_int, ctypes.POINTER(_Out)]
        L.cur_oracle_run.restype = ctypes.c_int
        L.cur_oracle_run_naive.argtypes = [vp, i64, i64, i64, dbl, i64, i64, vp, i64,
                                           ctypes.POINTER(_Out)]
        L.cur_oracle_run_naive.restype = ctypes.c_int
        L.cur_oracle_true_error.argtypes = [vp, i64, i64, i64, vp, vp, i64, vp]
        L.cur_oracle_true_error.restype = dbl
        L.cur_oracle_run_sketched.argtypes = [vp, vp, i64, i64, i64, dbl, i64, i64, u64, vp,
                                              i64, ctypes.c_int, ctypes.POINTER(_Out)]
        L.cur_oracle_run_sketched.restype = ctypes.c_int
        L.cur_oracle_gaussian_sketch_q8.argtypes = [u64, i64, i64, vp]
        L.cur_oracle_fixed_point.argtypes = [vp, i64, i64, i64, ctypes.c_int, vp]
        L.cur_oracle_quantize_q8.argtypes = [vp, i64, vp]
        L.cur_oracle_fixed_point_digits.argtypes = [dbl, ctypes.c_int, ctypes.c_int, vp]
        L.cur_oracle_sketch_fx.argtypes = [vp, i64, vp, i64, i64, i64, ctypes.c_int, vp]
        L.cur_oracle_run_y.argtypes = [vp, i64, i64, i64, dbl, i64, i64, vp, i64,
                                       ctypes.c_int, ctypes.POINTER(_Out)]
        L.cur_oracle_run_y.restype = ctypes.c_int
        L.cur_oracle_set_threads.argtypes = [ctypes.c_int]
        L.cur_oracle_threads.restype = ctypes.c_int
        L.cur_oracle_risk_threshold.argtypes = [dbl, dbl, dbl, dbl]
        L.cur_oracle_risk_threshold.restype = dbl
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().cur_oracle_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def gaussian_sketch(seed: int, c: int, m: int) -> np.ndarray:
    G = np.empty((c, m), dtype=np.float64)
    lib().cur_oracle_gaussian_sketch(seed, c, m, _p(G))
    return G


def sketch(G: np.ndarray, A: np.ndarray) -> np.ndarray:
    G, A = _f64(G), _f64(A)
    c, m = G.shape
    m2, n = A.shape
    assert m == m2
    Y = np.empty((c, n), dtype=np.float64)
    lib().cur_oracle_sketch(_p(G), c, _p(A), m, n, n, _p(Y))
    return Y


def lupp(M: np.ndarray, steps: int, excluded: np.ndarray | None = None):
    """Pivot rows of M chosen by `steps` steps of LU with partial pivoting.

    Returns (pivots, min_gap); `excluded` (uint8, len p) is updated in place.
    """
    M = _f64(M)
    p, q = M.shape
    piv = np.full(steps, -1, dtype=np.int64)
    gap = np.zeros(1, dtype=np.float64)
    ex = None if excluded is None else excluded
    if ex is not None:
        assert ex.dtype == np.uint8 and ex.flags.c_contiguous
    rc = lib().cur_oracle_lupp(_p(M), p, q, q, steps, _p(ex), _p(piv), _p(gap))
    if rc != 0:
        raise ValueError("fewer eligible rows than steps")
    return piv, float(gap[0])


def qrcp_pinv(M: np.ndarray, thr: float = -1.0):
    """(X, rank, perm, rdiag): generalised inverse of M by pivoted QR."""
    M = _f64(M)
    p, q = M.shape
    X = np.zeros((q, p), dtype=np.float64)
    perm = np.zeros(q, dtype=np.int64)
    rdiag = np.zeros(max(min(p, q), 1), dtype=np.float64)
    k = lib().cur_oracle_qrcp_pinv(_p(M), p, q, q, thr, _p(X), _p(perm), _p(rdiag))
    return X, int(k), perm, rdiag[:min(p, q)]


@dataclass
class Result:
    I: np.ndarray
    J: np.ndarray
    U: np.ndarray
    rho: float
    rho_hist: np.ndarray
    gap_col: np.ndarray
    gap_row: np.ndarray
    scale_row: np.ndarray
    rank: int
    iters: int
    normY: float
    maxabsY: float
    status: int
    S_final: np.ndarray | None


def _alloc_out(m, n, c, b, max_rank, want_S):
    R = max_rank
    K = (R + b - 1) // b + 2
    bufs = dict(I=np.full(R, -1, np.int64), J=np.full(R, -1, np.int64),
                U=np.zeros(R * R + 1, np.float64), rho_hist=np.zeros(K), gap_col=np.zeros(K),
                gap_row=np.zeros(K), scale_row=np.zeros(K),
                S_final=np.zeros((c, n)) if want_S else None)
    o = _Out()
    for name in ("I", "J", "U", "rho_hist", "gap_col", "gap_row", "scale_row", "S_final"):
        setattr(o, name, _p(bufs[name]))
    o.hist_cap = K
    return o, bufs


def _result(o, bufs) -> Result:
    r, k = int(o.rank), int(o.iters)
    return Result(I=bufs["I"][:r].copy(), J=bufs["J"][:r].copy(),
                  U=bufs["U"][:r * r].reshape(r, r).copy(), rho=float(o.rho),
                  rho_hist=bufs["rho_hist"][:k].copy(), gap_col=bufs["gap_col"][:k].copy(),
                  gap_row=bufs["gap_row"][:k].copy(), scale_row=bufs["scale_row"][:k].copy(),
                  rank=r, iters=k, normY=float(o.normY), maxabsY=float(o.maxabsY),
                  status=int(o.status), S_final=bufs["S_final"])


def run(A: np.ndarray, tol: float, b: int, c: int | None = None, seed: int = 0,
        G: np.ndarray | None = None, max_rank: int = 0, mode: int = 1,
        want_S: bool = False, A_sketch: np.ndarray | None = None) -> Result:
    """Algorithm 1 on A (FP64).  c defaults to floor(1.1 b) (Sec. 1.1).
    A_sketch (optional): the matrix the initial sketch is taken of."""
    A = _f64(A)
    m, n = A.shape
    if c is None:
        c = (11 * b) // 10
    R = min(m, n) if max_rank <= 0 else min(max_rank, m, n)
    if G is not None:
        G = _f64(G)
        assert G.shape == (c, m)
    o, bufs = _alloc_out(m, n, c, b, R, want_S)
    As = None if A_sketch is None else _f64(A_sketch)
    if As is not None:
        assert As.shape == A.shape
    rc = lib().cur_oracle_run_sketched(_p(A), _p(As), m, n, n, tol, b, c, seed, _p(G), R, mode,
                                       ctypes.byref(o))
    if rc != 0:
        raise ValueError("invalid arguments")
    return _result(o, bufs)


def run_naive(A: np.ndarray, tol: float, b: int, c: int, G: np.ndarray,
              max_rank: int = 0) -> Result:
    A, G = _f64(A), _f64(G)
    m, n = A.shape
    R = min(m, n) if max_rank <= 0 else min(max_rank, m, n)
    o, bufs = _alloc_out(m, n, c, b, R, False)
    lib().cur_oracle_run_naive(_p(A), m, n, n, tol, b, c, _p(G), R, ctypes.byref(o))
    return _result(o, bufs)


def true_error(A: np.ndarray, I, J, U) -> float:
    A = _f64(A)
    m, n = A.shape
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    U = _f64(U)
    r = len(I)
    return float(lib().cur_oracle_true_error(_p(A), m, n, n, _p(I), _p(J), r, _p(U)))


def risk_threshold(eps: float, delta: float, alpha: float, c: float) -> float:
    return float(lib().cur_oracle_risk_threshold(eps, delta, alpha, c))


def gaussian_sketch_q8(seed: int, c: int, m: int) -> np.ndarray:
    G = np.empty((c, m), dtype=np.float64)
    lib().cur_oracle_gaussian_sketch_q8(seed, c, m, _p(G))
    return G


def quantize_q8(G: np.ndarray) -> np.ndarray:
    """clamp(rint(16 G), -127, 127) of a given sketch (ties to even)."""
    G = _f64(G)
    out = np.empty_like(G)
    lib().cur_oracle_quantize_q8(_p(G), G.size, _p(out))
    return out


def fixed_point(A: np.ndarray, S: int) -> np.ndarray:
    A = _f64(A)
    m, n = A.shape
    out = np.empty_like(A)
    lib().cur_oracle_fixed_point(_p(A), m, n, n, S, _p(out))
    return out


def fixed_point_digits(x: float, E: int, S: int) -> np.ndarray:
    """The S digits of fix_S(x) at column scale 2^E, least significant first."""
    d = np.zeros(S, dtype=np.float64)
    lib().cur_oracle_fixed_point_digits(float(x), int(E), int(S), _p(d))
    return d


# The tensor-core FP64 form of the sketch: 52-bit fixed point per column.
FX_BITS = 52


def sketch_fx(Gq: np.ndarray, A: np.ndarray, Q: int = FX_BITS) -> np.ndarray:
    """Y = RN(Gq trunc(A 2^(Q-E_j))) 2^(E_j-Q), the integer sum exact."""
    Gq, A = _f64(Gq), _f64(A)
    c, m = Gq.shape
    m2, n = A.shape
    assert m == m2
    Y = np.empty((c, n), dtype=np.float64)
    lib().cur_oracle_sketch_fx(_p(Gq), c, _p(A), m, n, n, Q, _p(Y))
    return Y


def run_y(A: np.ndarray, tol: float, b: int, c: int, Y: np.ndarray, max_rank: int = 0,
          mode: int = 1, want_S: bool = False) -> Result:
    """Algorithm 1's loop on A from the given initial sketch Y (c x n)."""
    A, Y = _f64(A), _f64(Y)
    m, n = A.shape
    assert Y.shape == (c, n)
    R = min(m, n) if max_rank <= 0 else min(max_rank, m, n)
    o, bufs = _alloc_out(m, n, c, b, R, want_S)
    rc = lib().cur_oracle_run_y(_p(A), m, n, n, tol, b, c, _p(Y), R, mode, ctypes.byref(o))
    if rc != 0:
        raise ValueError("invalid arguments")
    return _result(o, bufs)


def run_fx(A: np.ndarray, tol: float, b: int, c: int, seed: int = 0, max_rank: int = 0,
           mode: int = 1, want_S: bool = False) -> Result:
    """The FP64 tensor-core form: the 8-bit sketch G_q of the seed and the exact
    52-bit fixed-point sketch, then Algorithm 1's loop in FP64."""
    A = _f64(A)
    Gq = gaussian_sketch_q8(seed, c, A.shape[0])
    return run_y(A, tol, b, c, sketch_fx(Gq, A), max_rank=max_rank, mode=mode, want_S=want_S)


def set_threads(n: int) -> None:
    """Host threads of the oracle's parallel loops (results do not change)."""
    lib().cur_oracle_set_threads(int(n))


def threads() -> int:
    return int(lib().cur_oracle_threads())
