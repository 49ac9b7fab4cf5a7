"""Column-block sharding of one IterativeCUR decomposition (arXiv 2509.21963,
Algorithm 1 in the Lemma 1 form of Sec. 3.2) over the ranks of a
torch.distributed process group.

Rank g holds the columns [col0_g, col0_g + n_g) of A (m x n_g), the same
columns of the sketched residual S^col and of the row factor R (Rt, r x n_g).
The index sets, the row residual, the cores and L are replicated.  Per
iteration k:

  * S^col is all-gathered (c x n) and every rank runs the same column LUPP
    (J_k, global indices);
  * A(:, J_k) and R(:, J_k) are assembled by a sum all-reduce of gathers in
    which each rank fills the columns it owns and writes 0.0 elsewhere: every
    entry has exactly one non-zero contribution, so the sum is exact;
  * S^row = A(:, J_k) - L R(:, J_k), the row LUPP (I_k), N = S^row(I_k, :),
    N^+ and L_k = S^row N^+ are computed on every rank;
  * R_k(:, own) = A(I_k, own) - L(I_k, :) R(:, own) and
    S^col(:, own) -= (S^col(:, J_k) N^+) R_k(:, own) stay local, and
    ||S^col||_F^2 is a sum all-reduce of the ranks' partial sums.

At exit A(I, J) is assembled like A(:, J_k) and U = A(I, J)^+ is formed on
every rank.  The communication per iteration is one all-gather of c n
doubles and all-reduces of b m + r b doubles plus one scalar.

The arithmetic of a rank goes through a backend object; CudaBackend runs the
library's C-ABI step kernels (cur_step_*) on the rank's GPU.  Without an
initialised process group the run uses a single rank.

With the FP64 tensor-core sketch (CudaBackend(sketch_mode=5)) every column of
Y = RN(G_q trunc(A 2^(52 - E_j))) 2^(E_j - 52) depends only on that column of
A (its own exponent E_j, an exact integer sum rounded once), so each rank's
block of S^col equals the same columns of the unsharded sketch bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EPS = 2.0 ** -52


@dataclass
class ShardResult:
    I: np.ndarray
    J: np.ndarray
    U: np.ndarray
    rank: int
    iterations: int
    rho: float
    status: int                       # 0: tol reached; CUR_TOL_UNREACHED (7): rank cap
    rho_history: list = field(default_factory=list)


def column_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Balanced contiguous column block [c0, c1) of rank `rank`."""
    return rank * n // world, (rank + 1) * n // world


class _Comm:
    """The collectives of a sharded run, on a backend's arrays."""

    def __init__(self, backend, group):
        import torch.distributed as dist
        self.dist = dist
        self.be = backend
        self.group = group
        self.active = dist.is_available() and dist.is_initialized()
        self.world = dist.get_world_size(group) if self.active else 1
        self.rank = dist.get_rank(group) if self.active else 0

    def allreduce_(self, x):
        if self.world > 1:
            t = self.be.comm_tensor(x)
            self.dist.all_reduce(t, group=self.group)
            self.be.comm_back(t, x)
        return x

    def allreduce_scalar(self, v: float) -> float:
        if self.world == 1:
            return v
        import torch
        t = self.be.comm_scalar(v)
        self.dist.all_reduce(t, group=self.group)
        return float(t.item())

    def allgather_cols(self, x, widths):
        """[x_0 | x_1 | ...] (rows x sum(widths)) from every rank's block."""
        if self.world == 1:
            return x
        import torch
        rows = x.shape[0]
        wmax = max(widths)
        t = self.be.comm_tensor(x)
        pad = torch.zeros((rows, wmax), dtype=t.dtype, device=t.device)
        pad[:, :t.shape[1]] = t
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(parts, pad, group=self.group)
        full = torch.cat([p[:, :w] for p, w in zip(parts, widths)], dim=1).contiguous()
        return self.be.from_comm(full)

    def allgather_int(self, v: int) -> list[int]:
        if self.world == 1:
            return [v]
        import torch
        t = self.be.comm_scalar(float(v))
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t, group=self.group)
        return [int(p.item()) for p in parts]


def run(backend, A_local, n: int, col0: int, tol: float, b: int, c: int, seed: int = 0,
        max_rank: int = 0, group=None) -> ShardResult:
    """IterativeCUR of the m x n matrix whose columns [col0, col0 + n_g) are
    A_local (m x n_g, this rank's block) on every rank of `group` (the same
    tol, b, c, seed and max_rank everywhere).  Every rank returns the same
    I, J and U."""
    comm = _Comm(backend, group)
    be = backend
    m, ng = A_local.shape
    if not (tol > 0.0) or b < 1 or c < b or m < 1 or n < 1:
        raise ValueError("need tol > 0, 1 <= b <= c, m, n >= 1")
    widths = comm.allgather_int(ng)
    if sum(widths) != n:
        raise ValueError("column blocks do not add up to n")
    mn = min(m, n)
    if max_rank <= 0 or max_rank > mn:
        max_rank = mn

    G = be.gaussian(seed, c, m)
    S, ss = be.sketch(G, A_local)                        # S^col(:, own), its ||.||^2
    nY = math.sqrt(comm.allreduce_scalar(ss))
    I = np.zeros(0, dtype=np.int64)
    J = np.zeros(0, dtype=np.int64)
    if nY == 0.0:   # G A = 0: nothing to approximate
        return ShardResult(I, J, np.zeros((0, 0)), 0, 0, 0.0, 0, [])
    LT = be.zeros((max_rank, m))                         # L^T, replicated
    Rt = be.zeros((max_rank, ng))                        # R(:, own)
    maskc, maskr = be.mask(n), be.mask(m)
    rho, r, k, thr_scale, hist = 1.0, 0, 0, None, []
    while rho > tol and r < max_rank:
        bk = min(b, max_rank - r)
        Sfull = comm.allgather_cols(S, widths)           # S^col, c x n
        Jk = be.lupp(Sfull, bk, maskc)                   # column LUPP (global indices)
        Jloc = be.shift(Jk, -col0)                       # outside [0, ng): not owned
        SrowT = comm.allreduce_(be.gather(A_local, bk, m, ridx=Jloc, trans=True))   # A(:,J_k)^T
        if r > 0:
            G1 = comm.allreduce_(be.gather(Rt[:r], r, bk, cidx=Jloc))               # R(:,J_k)
            be.gemm(-1.0, G1, LT[:r], beta=1.0, C=SrowT, out=SrowT, trans_a=True)
        Ik = be.lupp(SrowT, bk, maskr)                   # row LUPP
        N = be.gather(SrowT, bk, bk, ridx=Ik, trans=True)   # S^row(I_k, :)
        Rk = Rt[r:r + bk]
        be.gather(A_local, bk, ng, ridx=Ik, out=Rk)      # A(I_k, own)
        if r > 0:
            G2 = be.gather(LT[:r], r, bk, cidx=Ik)       # L(I_k, :)^T
            be.gemm(-1.0, G2, Rt[:r], beta=1.0, C=Rk, out=Rk, trans_a=True)
        if thr_scale is None:   # rank threshold: |R_00| of the first core, times 2^-52
            thr_scale = be.pinv_r00(N) * EPS
        Np = be.pinv(N, thr_scale * (r + bk))
        be.gemm(1.0, Np, SrowT, out=LT[r:r + bk], trans_a=True)   # L_k^T = N^+T S^row^T
        SJk = be.gather(Sfull, c, bk, cidx=Jk)
        T1 = be.gemm(1.0, SJk, Np)
        _, ssl = be.gemm(-1.0, T1, Rk, beta=1.0, C=S, out=S, sumsq=True)
        rho = math.sqrt(comm.allreduce_scalar(ssl)) / nY
        I = np.concatenate([I, be.to_numpy(Ik)])
        J = np.concatenate([J, be.to_numpy(Jk)])
        r += bk
        k += 1
        hist.append(rho)
    U = np.zeros((0, 0))
    if r > 0:
        Iv, Jv = be.index(I), be.shift(be.index(J), -col0)
        AIJ = comm.allreduce_(be.gather(A_local, r, r, ridx=Iv, cidx=Jv))
        U = be.to_numpy(be.pinv(AIJ, -1.0))
    return ShardResult(I, J, U, r, k, rho, 0 if rho <= tol else 7, hist)


class CudaBackend:
    """One rank's arithmetic on its GPU through the library's step kernels
    (Context.gaussian / sketch / lupp / gather / gemm / pinv).  Arrays are
    FP64 CUDA tensors; the process group is NCCL (or gloo, via host copies).
    sketch_mode 0: the FP64-pipe sketch; 5: the FP64 tensor-core sketch."""

    def __init__(self, ctx, nccl: bool = True, sketch_mode: int = 0):
        import torch
        if sketch_mode not in (0, 5):
            raise ValueError("sketch_mode must be 0 or 5")
        self.ctx = ctx
        self.torch = torch
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.nccl = nccl
        self.sketch_mode = sketch_mode

    def gaussian(self, seed, c, m):
        return self.ctx.gaussian(seed, c, m)

    def sketch(self, G, A):
        if self.sketch_mode == 5:
            if A.stride(0) % 2 or A.data_ptr() % 16:   # the tensor maps need an even pitch
                m, n = A.shape
                buf = self.torch.empty((m, n + 1), dtype=A.dtype, device=A.device)[:, :n]
                buf.copy_(A)
                A = buf
            return self.ctx.sketch_fx(G, A)
        return self.ctx.sketch(G, A)

    def zeros(self, shape):
        return self.torch.zeros(shape, dtype=self.torch.float64, device=self.dev)

    def mask(self, n):
        return self.torch.zeros(n, dtype=self.torch.uint8, device=self.dev)

    def index(self, idx):
        return self.torch.as_tensor(np.asarray(idx, dtype=np.int64), device=self.dev)

    def shift(self, idx, d):
        return idx + d

    def lupp(self, X, steps, mask):
        piv, _ = self.ctx.lupp(X, steps, mask)
        return piv

    def gather(self, X, rows, cols, ridx=None, cidx=None, trans=False, out=None):
        return self.ctx.gather(X, rows, cols, ridx=ridx, cidx=cidx, trans=trans, out=out)

    def gemm(self, alpha, A, B, beta=0.0, C=None, out=None, trans_a=False, trans_b=False,
             sumsq=False):
        return self.ctx.gemm(alpha, A, B, beta=beta, C=C, out=out, trans_a=trans_a,
                             trans_b=trans_b, sumsq=sumsq)

    def pinv(self, M, thr):
        X, _ = self.ctx.pinv(M, thr)
        return X

    def pinv_r00(self, M):
        # |R_00| of pivoted QR is the largest column norm of M
        Mh = M.cpu().numpy()
        return float(np.sqrt((Mh * Mh).sum(axis=0).max())) if Mh.size else 0.0

    def to_numpy(self, x):
        return x.cpu().numpy()

    def comm_tensor(self, x):
        return x if self.nccl else x.cpu()

    def comm_back(self, t, x):
        if t.data_ptr() != x.data_ptr():
            x.copy_(t)

    def comm_scalar(self, v):
        return self.torch.tensor([v], dtype=self.torch.float64,
                                 device=self.dev if self.nccl else "cpu")

    def from_comm(self, t):
        return t.to(self.dev)
