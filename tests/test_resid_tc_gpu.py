"""Residual products of the loop on the tensor cores (cur_opts.residual_planes,
cur_step_resid_tc): D(n, i) -= sum_k P(i, k) Q(n, k) with P and Q split into
2 or 3 BF16 planes and FP32 accumulation.

Bound used (derived from the arithmetic): a BF16 plane keeps 8 significant
bits with round-to-nearest (unit roundoff 2^-8), so x = x_0 + ... +
x_{NP-1} + e with |e| <= 2^-(8 NP) |x| and |x_a| <= 2^-(8 a) (1 + 2^-8) |x|;
the products keep the plane pairs (a, b) with a + b < NP, so the dropped pairs
and the two representation errors stay below 4 NP 2^-(8 NP) |x||y|; BF16
products are exact in FP32 and every one of the NM = NP (NP + 1) / 2 MMAs per
K step adds into one FP32 accumulator, so the sums add at most
NM K 2^-24 sum_k |P(i, k) Q(n, k)| (the usual gamma bound).  So
|D_gpu - D_exact| <= (4 NP 2^-(8 NP) + 1.01 NM K 2^-24) sum_k |P(i,k)||Q(n,k)|.
(The sums inside one MMA need not round like a sequence of FP32 additions;
measured, a third plane improves a 200-term product only ~3x over two, while
a single product improves by the full 2^8.)  Whole runs in this form are
compared with the oracle run on the same sketch
over the selections whose oracle gaps exceed the product error, and must
reach the tolerance with a CUR as accurate as the FP64 loop's.
"""
import numpy as np
import pytest

import oracle
from paper_2509_21963_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_parity_gpu import _decided_prefix  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_21963_gb300 as cur
    c = cur.Context(0)
    yield c
    c.close()


def _bound(P, Q, planes):
    nm = planes * (planes + 1) // 2
    K = P.shape[1]
    c = 4 * planes * 2.0 ** (-8 * planes) + 1.01 * nm * K * 2.0 ** -24
    return c * (np.abs(Q) @ np.abs(P).T)


@pytest.mark.parametrize("planes", [2, 3])
@pytest.mark.parametrize("M,N,K", [(300, 50, 200), (1000, 128, 64), (129, 1, 1), (257, 7, 1000),
                                   (4000, 100, 130)])
def test_resid_tc_step_within_bound(ctx, planes, M, N, K):
    rng = np.random.default_rng(M + N + K + planes)
    P = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, size=(M, 1)))
    Q = rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, size=(1, K)))
    D = rng.standard_normal((N, M))
    Dd = torch.from_numpy(D.copy()).cuda()
    ctx.resid_tc(torch.from_numpy(P).cuda(), torch.from_numpy(Q).cuda(), Dd, planes)
    exact = D - Q @ P.T
    err = np.abs(Dd.cpu().numpy() - exact)
    assert np.all(err <= _bound(P, Q, planes)), err.max()
    if planes == 3 and K == 1:
        # with a single product there are no sums: the third plane must take the
        # error from the two-plane level (~2^-16) to ~2^-24 of |P||Q|
        D2 = torch.from_numpy(D.copy()).cuda()
        ctx.resid_tc(torch.from_numpy(P).cuda(), torch.from_numpy(Q).cuda(), D2, 2)
        err2 = np.abs(D2.cpu().numpy() - exact)
        assert err.max() <= 0.05 * err2.max(), (err.max(), err2.max())


def test_resid_tc_strided_and_zero_k(ctx):
    rng = np.random.default_rng(3)
    Pf = rng.standard_normal((500, 96))
    Qf = rng.standard_normal((40, 80))
    P, Q = Pf[:, :70], Qf[:, :70]
    D = rng.standard_normal((40, 520))
    Dd = torch.from_numpy(D.copy()).cuda()
    ctx.resid_tc(torch.from_numpy(Pf).cuda()[:, :70], torch.from_numpy(Qf).cuda()[:, :70],
                 Dd[:, :500], 2)
    got = Dd.cpu().numpy()
    assert np.all(np.abs(got[:, :500] - (D[:, :500] - Q @ P.T)) <= _bound(P, Q, 2))
    assert np.array_equal(got[:, 500:], D[:, 500:])       # columns past M untouched
    Dd = torch.from_numpy(D.copy()).cuda()
    ctx.resid_tc(torch.zeros(500, 0, dtype=torch.float64).cuda(),
                 torch.zeros(40, 0, dtype=torch.float64).cuda(), Dd, 3)
    assert np.array_equal(Dd.cpu().numpy(), D)


@pytest.mark.parametrize("S,tol,planes", [(2, 1e-3, 2), (2, 1e-4, 3), (3, 1e-5, 3)])
def test_resid_tc_run(ctx, S, tol, planes):
    """1000 x 800 FP32 (s_i = 10^(-i/50)), b = 10, c = 30, the S-digit sketch:
    the run with the residual products on the tensor cores selects the oracle's
    indices wherever the oracle's LUPP gaps exceed the product error, reaches
    the tolerance, and its CUR is as accurate as the FP64 loop's.  (Tol 1e-6 is
    below this form's floor: with three planes rho stalls at 1.9e-6 at full
    rank on this matrix.)"""
    A32 = inputs.cfg_small(S).astype(np.float32)
    A = A32.astype(np.float64)
    Ad = torch.from_numpy(A32).cuda()
    Gq = oracle.gaussian_sketch_q8(S, 30, 1000)
    ref = oracle.run(A, tol, 10, 30, G=Gq, mode=1, A_sketch=oracle.fixed_point(A, S))
    got = ctx.run(Ad, tol, 10, 30, S, sketch_mode=S, residual_planes=planes)
    tau = {2: 1e-3, 3: 1e-5}[planes]
    n_dec = _decided_prefix(ref, 10, ref.maxabsY, tau)
    assert n_dec >= 10
    assert np.array_equal(got.I[:n_dec], ref.I[:n_dec])
    assert np.array_equal(got.J[:n_dec], ref.J[:n_dec])
    assert got.status == 0 and got.rho <= tol
    plain = ctx.run(Ad, tol, 10, 30, S, sketch_mode=S)
    err = oracle.true_error(A, got.I, got.J, got.U)
    err_plain = oracle.true_error(A, plain.I, plain.J, plain.U)
    assert err <= max(tol, 1.25 * err_plain), (err, err_plain)


def test_resid_tc_argument_errors(ctx):
    import paper_2509_21963_gb300 as cur
    A = torch.zeros(300, 300, dtype=torch.float32, device="cuda")
    for kw, b, c in [(dict(residual_planes=1), 8, 9), (dict(residual_planes=4), 8, 9),
                     (dict(residual_planes=2), 130, 143)]:
        with pytest.raises(cur.CurError) as e:
            ctx.run(A, 1e-3, b, c, 0, sketch_mode=2, **kw)
        assert e.value.status == cur.CUR_EINVAL
    with pytest.raises(cur.CurError) as e:
        ctx.resid_tc(torch.zeros(10, 4, dtype=torch.float64).cuda(),
                     torch.zeros(129, 4, dtype=torch.float64).cuda(),
                     torch.zeros(129, 10, dtype=torch.float64).cuda(), 2)
    assert e.value.status == cur.CUR_EINVAL
