"""Column-block sharding of one decomposition (paper_2509_21963_gb300.shard)
on CPU ranks (gloo).  The ranks' arithmetic is the FP64 oracle's: the
gaussian sketch, the sketch, LUPP and pivoted QR are the oracle's own
functions, and the products are sums in the oracle's order (sequential over
the inner index, multiply then add), so the sharded run must return the
oracle's I, J and U exactly; world size 2 must equal world size 1 bit for
bit (only ||S^col||_F^2 is summed in another order, so rho agrees to
rounding)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2509_21963_gb300 import inputs, shard

torch = pytest.importorskip("torch")


class OracleBackend:
    """Test stand-in for a rank's device: numpy arrays, oracle arithmetic.
    fx: the sketch is the oracle's exact 52-bit fixed-point form (G_q from G)."""

    def __init__(self, fx=False):
        self.fx = fx

    def gaussian(self, seed, c, m):
        return oracle.gaussian_sketch(seed, c, m)

    def sketch(self, G, A):
        if self.fx:
            Y = oracle.sketch_fx(oracle.quantize_q8(G), np.ascontiguousarray(A))
        else:
            Y = oracle.sketch(G, np.ascontiguousarray(A))
        return Y, float((Y * Y).sum())

    def zeros(self, shape):
        return np.zeros(shape)

    def mask(self, n):
        return np.zeros(n, dtype=np.uint8)

    def index(self, idx):
        return np.asarray(idx, dtype=np.int64)

    def shift(self, idx, d):
        return idx + d

    def lupp(self, X, steps, mask):     # candidates: the columns of X
        piv, _ = oracle.lupp(np.ascontiguousarray(X.T), steps, mask)
        return piv

    def gather(self, X, rows, cols, ridx=None, cidx=None, trans=False, out=None):
        Xv = X.T if trans else X
        r = np.arange(rows) if ridx is None else np.asarray(ridx)
        c = np.arange(cols) if cidx is None else np.asarray(cidx)
        rok = (r >= 0) & (r < Xv.shape[0])
        cok = (c >= 0) & (c < Xv.shape[1])
        res = np.zeros((rows, cols))
        res[np.ix_(rok, cok)] = Xv[np.ix_(r[rok], c[cok])]
        if out is None:
            return res
        out[...] = res
        return out

    def gemm(self, alpha, A, B, beta=0.0, C=None, out=None, trans_a=False, trans_b=False,
             sumsq=False):
        Aop = A.T if trans_a else A
        Bop = B.T if trans_b else B
        s = np.zeros((Aop.shape[0], Bop.shape[1]))
        for k in range(Aop.shape[1]):   # the oracle's order: s = s + a * b, k ascending
            s = s + Aop[:, k:k + 1] * Bop[k:k + 1, :]
        if beta == 0.0:
            D = s if alpha == 1.0 else alpha * s
        elif beta == 1.0 and alpha == -1.0:
            D = C - s
        else:
            D = beta * C + alpha * s
        if out is not None:
            out[...] = D
            D = out
        return (D, float((D * D).sum())) if sumsq else D

    def pinv(self, M, thr):
        return oracle.qrcp_pinv(M, thr)[0]

    def pinv_r00(self, M):
        return abs(oracle.qrcp_pinv(M, -1.0)[3][0])

    def to_numpy(self, x):
        return np.asarray(x)

    def comm_tensor(self, x):
        return torch.from_numpy(np.ascontiguousarray(x))

    def comm_back(self, t, x):
        x[...] = t.numpy()

    def comm_scalar(self, v):
        return torch.tensor([v], dtype=torch.float64)

    def from_comm(self, t):
        return t.numpy()


CASES = {
    "small": (lambda: inputs.cfg_small(0), 1e-6, 10, 30, 0),
    "odd": (lambda: inputs.svd_matrix(300, 257, 0.9 ** np.arange(257), seed=3), 1e-8, 7, 12, 4),
    "fx": (lambda: inputs.svd_matrix(400, 301, 0.85 ** np.arange(301), seed=6), 1e-8, 9, 14, 2),
}


def _run(case, world=1, rank=0, group=None):
    make, tol, b, c, seed = CASES[case]
    A = make()
    n = A.shape[1]
    c0, c1 = shard.column_range(n, world, rank)
    return shard.run(OracleBackend(fx=case == "fx"), np.ascontiguousarray(A[:, c0:c1]), n, c0,
                     tol, b, c, seed, group=group)


def test_fx_sketch_blocks_equal_columns():
    """The exact fixed-point sketch of a column block is the same columns of
    the whole matrix's sketch, bit for bit, and the seeded 8-bit sketch is the
    rounding of the seeded Gaussian."""
    A = CASES["fx"][0]()
    Gq = oracle.quantize_q8(oracle.gaussian_sketch(2, 14, A.shape[0]))
    assert np.array_equal(Gq, oracle.gaussian_sketch_q8(2, 14, A.shape[0]))
    Y = oracle.sketch_fx(Gq, A)
    for c0, c1 in [(0, 150), (150, 301), (7, 8)]:
        assert np.array_equal(oracle.sketch_fx(Gq, np.ascontiguousarray(A[:, c0:c1])), Y[:, c0:c1])


@pytest.mark.parametrize("case", list(CASES))
def test_single_rank_equals_oracle(case):
    make, tol, b, c, seed = CASES[case]
    A = make()
    if case == "fx":
        ref = oracle.run_fx(A, tol, b, c, seed=seed, mode=1)
    else:
        ref = oracle.run(A, tol, b, c, seed=seed, mode=1)
    got = _run(case)
    assert got.rank == ref.rank and got.status == ref.status
    assert np.array_equal(got.I, ref.I) and np.array_equal(got.J, ref.J)
    assert np.array_equal(got.U, ref.U.reshape(got.U.shape))
    np.testing.assert_allclose(got.rho_history, ref.rho_hist[:len(got.rho_history)],
                               rtol=1e-12)


def test_column_ranges_cover():
    for n, w in [(800, 2), (257, 2), (10, 3), (5, 4)]:
        rs = [shard.column_range(n, w, g) for g in range(w)]
        assert rs[0][0] == 0 and rs[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = _run(case, world, rank)
        q.put((rank, r.I, r.J, r.U, r.rho_history, r.status))
    finally:
        dist.destroy_process_group()


def _spawn_ranks(case, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, *rest = q.get(timeout=300)
        out[rank] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("case", ["odd", "fx"])
def test_three_ranks_equal_one(case):
    """World size 3 (gloo): blocks of 85/86/86 (n = 257) and 100/100/101
    (n = 301) columns; every rank returns the single-rank I, J and U."""
    out = _spawn_ranks(case, 3)
    one = _run(case)
    for rank in range(3):
        I, J, U, hist, status = out[rank]
        assert np.array_equal(I, one.I) and np.array_equal(J, one.J)
        assert np.array_equal(U, one.U)
        assert status == one.status
        np.testing.assert_allclose(hist, one.rho_history, rtol=1e-12)


@pytest.mark.parametrize("case", list(CASES))
def test_two_ranks_equal_one(case):
    """World size 2 (gloo): both ranks return the single-rank I, J and U bit
    for bit; the column blocks are [0, n/2) and [n/2, n) (uneven for n odd)."""
    out = _spawn_ranks(case, 2)
    one = _run(case)
    for rank in (0, 1):
        I, J, U, hist, status = out[rank]
        assert np.array_equal(I, one.I) and np.array_equal(J, one.J)
        assert np.array_equal(U, one.U)
        assert status == one.status
        np.testing.assert_allclose(hist, one.rho_history, rtol=1e-12)
