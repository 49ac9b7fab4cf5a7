"""The sharded run on the GPU step kernels (CudaBackend, one rank): it makes
the same kernel calls in the same order as cur_run, so I, J, U and rho equal
cur_run's bit for bit.  Also the two step entry points it adds to the C ABI
(cur_step_gemm, cur_step_gather) against plain PyTorch FP64 on the CPU."""
import numpy as np
import pytest

import oracle
from paper_2509_21963_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_21963_gb300 as cur
    c = cur.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("trans_a,trans_b", [(False, False), (True, False), (False, True),
                                             (True, True)])
def test_step_gemm_matches_torch(ctx, trans_a, trans_b):
    rng = np.random.default_rng(int(trans_a) * 2 + int(trans_b))
    M, N, K = 37, 301, 19
    A = rng.standard_normal((K, M) if trans_a else (M, K))
    B = rng.standard_normal((N, K) if trans_b else (K, N))
    C = rng.standard_normal((M, N))
    Ad, Bd, Cd = (torch.from_numpy(x).cuda() for x in (A, B, C))
    D, ss = ctx.gemm(-0.5, Ad, Bd, beta=2.0, C=Cd, trans_a=trans_a, trans_b=trans_b, sumsq=True)
    ref = -0.5 * torch.from_numpy(A.T if trans_a else A) @ torch.from_numpy(B.T if trans_b else B) \
        + 2.0 * torch.from_numpy(C)
    D = D.cpu()
    # |error| <= K u (|alpha| |A||B| + |beta C|) per entry, u = 2^-53
    bound = (K + 2) * 2.0 ** -53 * (0.5 * np.abs(A.T if trans_a else A) @ np.abs(B.T if trans_b else B)
                                    + 2.0 * np.abs(C))
    assert np.all(np.abs((D - ref).numpy()) <= bound)
    assert abs(ss - float((D * D).sum())) <= 1e-12 * ss
    # in place (C aliases D), beta = 0 ignores C
    ctx.gemm(1.0, Ad, Bd, beta=1.0, C=Cd, out=Cd, trans_a=trans_a, trans_b=trans_b)
    D0 = ctx.gemm(1.0, Ad, Bd, trans_a=trans_a, trans_b=trans_b)
    assert torch.allclose(Cd.cpu(), torch.from_numpy(C) + D0.cpu(), rtol=0, atol=1e-12)


def test_step_gather_bounds(ctx):
    X = torch.arange(35, dtype=torch.float64).reshape(5, 7).cuda()
    ridx = torch.tensor([4, -1, 0, 5], dtype=torch.int64).cuda()
    cidx = torch.tensor([6, 0, 7], dtype=torch.int64).cuda()
    out = ctx.gather(X, 4, 3, ridx=ridx, cidx=cidx).cpu().numpy()
    Xh = X.cpu().numpy()
    exp = np.zeros((4, 3))
    for a, r in enumerate([4, -1, 0, 5]):
        for t, c in enumerate([6, 0, 7]):
            if 0 <= r < 5 and 0 <= c < 7:
                exp[a, t] = Xh[r, c]
    assert np.array_equal(out, exp)
    outT = ctx.gather(X, 2, 5, ridx=torch.tensor([6, 1], dtype=torch.int64).cuda(), trans=True)
    assert np.array_equal(outT.cpu().numpy(), Xh[:, [6, 1]].T)


@pytest.mark.parametrize("case", ["small", "exact_rank"])
def test_single_rank_shard_equals_cur_run(ctx, case):
    from paper_2509_21963_gb300 import shard
    if case == "small":
        A, tol, b, c, seed = inputs.cfg_small(0), 1e-6, 10, 30, 0
    else:
        A, tol, b, c, seed = inputs.exact_rank(500, 400, 37, seed=4), 1e-10, 10, 30, 2
    Ad = torch.from_numpy(A).cuda()
    ref = ctx.run(Ad, tol, b, c, seed)
    got = shard.run(shard.CudaBackend(ctx), Ad, A.shape[1], 0, tol, b, c, seed)
    assert got.rank == ref.rank and got.status == ref.status
    assert np.array_equal(got.I, ref.I) and np.array_equal(got.J, ref.J)
    assert np.array_equal(got.U, ref.U.reshape(got.U.shape))
    assert got.rho == ref.rho
    assert oracle.true_error(A, got.I, got.J, got.U) <= 10 * tol


@pytest.mark.parametrize("case", ["small", "exact_rank"])
def test_single_rank_shard_fx_equals_cur_run(ctx, case):
    """With the FP64 tensor-core sketch (CudaBackend(sketch_mode=5)) the
    sharded run makes cur_run's calls with sketch_mode 5 (G from the seed, the
    exact fixed-point sketch, then the FP64 loop): the same I, J, U and rho."""
    from paper_2509_21963_gb300 import shard
    if case == "small":
        A, tol, b, c, seed = inputs.cfg_small(0), 1e-6, 10, 30, 0
    else:
        A, tol, b, c, seed = inputs.exact_rank(500, 400, 37, seed=4), 1e-10, 10, 30, 2
    Ad = torch.from_numpy(A).cuda()
    ref = ctx.run(Ad, tol, b, c, seed, sketch_mode=5)
    got = shard.run(shard.CudaBackend(ctx, sketch_mode=5), Ad, A.shape[1], 0, tol, b, c, seed)
    assert got.rank == ref.rank and got.status == ref.status
    assert np.array_equal(got.I, ref.I) and np.array_equal(got.J, ref.J)
    assert np.array_equal(got.U, ref.U.reshape(got.U.shape))
    assert got.rho == ref.rho


def test_shard_fx_odd_width_block(ctx):
    """An odd-width column block (odd row pitch) is copied to an even pitch for
    the tensor maps; the run then selects the oracle's indices (exact sketch,
    FP64 loop) wherever the oracle's LUPP gaps are above rounding, and its CUR
    is as accurate as the oracle's (the 135 x 135 core has entries ~1e9, so U
    itself agrees only to its conditioning; the true error, ~3.4e-7, is well
    above tol: rho is the sketched estimate)."""
    from paper_2509_21963_gb300 import shard
    from test_parity_gpu import _decided_prefix
    A = inputs.svd_matrix(400, 301, 0.85 ** np.arange(301), seed=6)
    tol, b, c, seed = 1e-8, 9, 14, 2
    got = shard.run(shard.CudaBackend(ctx, sketch_mode=5), torch.from_numpy(A).cuda(), 301, 0,
                    tol, b, c, seed)
    ref = oracle.run_fx(A, tol, b, c, seed=seed, mode=1)
    n_dec = _decided_prefix(ref, b, ref.maxabsY)
    assert n_dec >= b
    assert np.array_equal(got.I[:n_dec], ref.I[:n_dec]) and np.array_equal(got.J[:n_dec], ref.J[:n_dec])
    err_ref = oracle.true_error(A, ref.I, ref.J, ref.U)
    assert oracle.true_error(A, got.I, got.J, got.U) <= 2 * err_ref
