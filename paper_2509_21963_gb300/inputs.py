"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds no arithmetic of the method: it only builds matrices (and,
for tests, explicit Gaussian sketches) from seeds.  Both the CUDA path and the
CPU oracle consume what it produces.

Workloads (Sec. 5 of arXiv 2509.21963 uses SuiteSparse and Gaussian-product
matrices; these synthetic stand-ins keep their sizes and spectra):
  * ``svd_matrix``        A = U diag(s) V^T, U, V Haar-orthogonal (QR of a Gaussian
                          with the sign fix of Mezzadri 2007), any spectrum s.
  * ``exact_rank``        A = X Y^T with Gaussian X, Y (rank r exactly).
  * ``low_rank_gaussian`` the paper's Low-Rank matrix G1 G2^T (Sec. 5.1).
  * ``lehmer``            A_ij = min(i,j)/max(i,j) (Sec. 5.3).
  * ``decay_matrix_torch`` large matrices built on the GPU with torch (thin
                          orthonormal factors of a capped rank plus i.i.d. noise).
  * ``batch_specs`` / ``batch_matrix`` / ``batch_matrix_torch``  the many-small-
                          matrices workload: m, n log-uniform, spectrum drawn from
                          {exp(-i/20), i^-1.5, exact rank r ~ U[5, 200] with unit
                          singular values}.
"""
from __future__ import annotations

import numpy as np


def haar_orthogonal(n: int, k: int, rng: np.random.Generator) -> np.ndarray:
    """n x k matrix with orthonormal columns, Haar distributed (k <= n)."""
    Z = rng.standard_normal((n, k))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def svd_matrix(m: int, n: int, s: np.ndarray, seed: int) -> np.ndarray:
    """A = U diag(s) V^T with Haar U (m x k), V (n x k), k = len(s)."""
    rng = np.random.default_rng(seed)
    k = len(s)
    U = haar_orthogonal(m, k, rng)
    V = haar_orthogonal(n, k, rng)
    return (U * np.asarray(s, dtype=np.float64)) @ V.T


def cfg_small(seed: int = 0) -> np.ndarray:
    """1000 x 800, s_i = 10^(-i/50), i = 1..800 (the small parity workload)."""
    s = 10.0 ** (-np.arange(1, 801) / 50.0)
    return svd_matrix(1000, 800, s, seed)


def exact_rank(m: int, n: int, r: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, r)) @ rng.standard_normal((n, r)).T


def low_rank_gaussian(m: int, n: int, r: int, seed: int) -> np.ndarray:
    """The Low-Rank test matrix of Sec. 5.1: G1 G2^T with standard Gaussians."""
    return exact_rank(m, n, r, seed)


def lehmer(n: int) -> np.ndarray:
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.minimum.outer(i, i) / np.maximum.outer(i, i)


def explicit_sketch(c: int, m: int, seed: int) -> np.ndarray:
    """An explicit Gaussian sketch (c x m), for tests that pass G as an input."""
    return np.random.default_rng(seed + 7919).standard_normal((c, m))


def decay_matrix_torch(m: int, n: int, spectrum: str, seed: int, noise: float = 0.0,
                       rank_cap: int = 2000, dtype=None, device="cuda", factor_dtype=None):
    """Large A = U_k diag(s_1..s_k) V_k^T + noise * N(0,1), built with torch.

    U_k, V_k: thin Q factors of seeded Gaussians (k = rank_cap columns).  By
    default the factors and their product run in FP32 (rounding ~1e-7 per
    operation, which accumulates to ~3e-5 of ||A|| over k = 4096 terms: far
    below the noise term of the noisy workloads); factor_dtype=torch.float64
    keeps the construction exact to FP64 for noise-free matrices whose small
    tolerances must be reachable.  The noise is drawn and added in FP64 before
    the final cast to ``dtype``.
    spectrum: "poly2" (i^-2), "exp200" (exp(-i/200)), "exp20" (exp(-i/20)),
              "poly1.5" (i^-1.5).
    """
    import torch
    dtype = dtype or torch.float64
    k = min(rank_cap, m, n)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    i = torch.arange(1, k + 1, device=device, dtype=torch.float64)
    if spectrum == "poly2":
        s = i ** -2.0
    elif spectrum == "poly1.5":
        s = i ** -1.5
    elif spectrum == "exp200":
        s = torch.exp(-i / 200.0)
    elif spectrum == "exp20":
        s = torch.exp(-i / 20.0)
    else:
        raise ValueError(spectrum)
    fd = factor_dtype or torch.float32
    U = torch.linalg.qr(torch.randn(m, k, device=device, generator=g, dtype=torch.float32).to(fd))[0]
    V = torch.linalg.qr(torch.randn(n, k, device=device, generator=g, dtype=torch.float32).to(fd))[0]
    A = torch.empty(m, n, device=device, dtype=dtype)
    rows = max(1, (1 << 27) // max(n, 1))
    for r0 in range(0, m, rows):
        r1 = min(m, r0 + rows)
        blk = ((U[r0:r1] * s.to(fd)) @ V.T).to(torch.float64)
        if noise > 0.0:
            blk += noise * torch.randn(r1 - r0, n, device=device, generator=g, dtype=torch.float64)
        A[r0:r1] = blk.to(dtype)
    del U, V
    return A


def low_rank_gaussian_torch(m: int, n: int, r: int, seed: int, device="cuda"):
    """The Low-Rank matrix of Sec. 5.1 built on the GPU in FP64: G1 G2^T with
    standard Gaussian G1 (m x r), G2 (n x r), so its rank is exactly r."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G1 = torch.randn(m, r, device=device, generator=g, dtype=torch.float64)
    G2 = torch.randn(n, r, device=device, generator=g, dtype=torch.float64)
    A = G1 @ G2.T
    del G1, G2
    return A


BATCH_KINDS = ("exp20", "poly1.5", "rank")


def batch_specs(njobs: int, seed: int, lo: int = 64, hi: int = 2048):
    """Shapes and spectra of a batch: m, n log-uniform in [lo, hi], kind uniform
    over BATCH_KINDS, exact rank r ~ U[5, 200]; one matrix seed per job."""
    rng = np.random.default_rng(seed)
    lg = lambda: np.exp(rng.uniform(np.log(lo), np.log(hi + 1), njobs))  # noqa: E731
    m = np.clip(lg().astype(np.int64), lo, hi)
    n = np.clip(lg().astype(np.int64), lo, hi)
    kind = rng.integers(0, 3, njobs)
    r = rng.integers(5, 201, njobs)
    return [dict(m=int(m[j]), n=int(n[j]), kind=BATCH_KINDS[kind[j]], r=int(r[j]),
                 seed=int(seed * 100003 + j)) for j in range(njobs)]


def batch_spectrum(m: int, n: int, kind: str, r: int) -> np.ndarray:
    k = min(m, n)
    i = np.arange(1, k + 1, dtype=np.float64)
    if kind == "exp20":
        return np.exp(-i[: min(k, 800)] / 20.0)   # e^-40: below FP64 rounding of s_1
    if kind == "poly1.5":
        return i ** -1.5
    if kind == "rank":
        return np.ones(min(r, k))
    raise ValueError(kind)


def batch_matrix(spec: dict) -> np.ndarray:
    """FP64 A = U diag(s) V^T with Haar factors for one batch job (numpy)."""
    return svd_matrix(spec["m"], spec["n"], batch_spectrum(spec["m"], spec["n"], spec["kind"],
                                                           spec["r"]), spec["seed"])


def batch_matrix_torch(spec: dict, dtype=None, device="cuda"):
    """The same recipe on the GPU with torch (orthonormal factors from the QR of
    seeded Gaussians; not the numpy matrix of the same spec).  Factors and
    product in FP32 (TF32 off): orthonormal to ~1e-7, so the singular values
    are s_i (1 + O(1e-7)), below the FP32 rounding of the stored entries."""
    import torch
    dtype = dtype or torch.float32
    s = torch.from_numpy(batch_spectrum(spec["m"], spec["n"], spec["kind"], spec["r"]))
    s = s.to(device=device, dtype=torch.float32)
    k = s.numel()
    g = torch.Generator(device=device)
    g.manual_seed(spec["seed"])
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        U = torch.linalg.qr(torch.randn(spec["m"], k, device=device, generator=g))[0]
        V = torch.linalg.qr(torch.randn(spec["n"], k, device=device, generator=g))[0]
        A = (U * s) @ V.T
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return A.to(dtype).contiguous()
