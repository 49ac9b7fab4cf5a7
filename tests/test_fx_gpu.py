"""GPU parity of the FP64 tensor-core form (CUR_SKETCH_F64_TC) against the oracle.

The sketch is exact by construction: Y = RN(G_q trunc(A 2^(52-E_j))) 2^(E_j-52)
with the integer sum formed exactly and rounded once, which the oracle
(``oracle.sketch_fx``) evaluates with 128-bit integers.  So the sketch is
compared bit for bit; the runs then follow the plain method's gates (I, J
bit-exact where the oracle's decisions are not at rounding level, rho and U as
in test_parity_gpu.py), with the oracle started from its own exact sketch
(``oracle.run_fx``).
"""
import numpy as np
import pytest

import oracle
from paper_2509_21963_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_parity_gpu import _check_parity  # noqa: E402  (same gates as the plain form)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_21963_gb300 as cur
    c = cur.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _hard_matrix(m, n, seed):
    """Gaussian entries with columns of special structure: zero, wide dynamic
    range, exact power-of-two maximum, subnormals inside a normal column, a
    column of subnormals only, huge values, negative zeros."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    if n >= 8:
        A[:, 1] = 0.0
        A[:, 2] *= 10.0 ** rng.uniform(-12, 3, m)
        A[:, 3] = rng.uniform(-511, 511, m)
        A[0, 3] = 512.0
        A[:3, 4] = [5e-324, -1e-310, 2.5e-308]
        A[:, 5] = rng.uniform(-1e-309, 1e-309, m)
        A[:, 6] *= 2.0 ** 900
        A[::3, 7] = -0.0
    return A


@pytest.mark.parametrize("c,m,n", [                # n even: the row stride feeds TMA
    (55, 2048, 1998),     # ragged column strip, 4 chunks
    (30, 1000, 800),      # the small workload's shape
    (7, 333, 66),         # c pads to 16; rows not a multiple of 16; one strip
    (64, 4097, 130),      # N = 64, one row past a chunk, 2 columns in the last strip
    (140, 517, 334),      # three row groups of G (64, 64, 12)
    (1, 16, 2),           # minimal
])
def test_sketch_fx_bit_exact(ctx, c, m, n):
    A = _hard_matrix(m, n, seed=m + n + c)
    G = oracle.gaussian_sketch(4, c, m)
    Y, ss = ctx.sketch_fx(dev(G), dev(A))
    Yo = oracle.sketch_fx(oracle.quantize_q8(G), A)
    np.testing.assert_array_equal(Y.cpu().numpy(), Yo)
    with np.errstate(over="ignore"):
        so = (Yo ** 2).sum()           # the 2^900 column overflows ||Y||^2 on both sides
    assert ss == so if not np.isfinite(so) else abs(ss - so) <= 1e-12 * so


def test_sketch_fx_strides_and_nonfinite(ctx):
    """An even row stride larger than n; a column with Inf (NaN in Y); odd
    stride and misaligned base are rejected with CUR_EINVAL."""
    import paper_2509_21963_gb300 as cur
    m, n, c = 700, 301, 20
    rng = np.random.default_rng(5)
    Afull = rng.standard_normal((m, n + 2))
    Ad = dev(Afull)[:, :n]                     # stride n + 2 = 303 (odd): rejected
    G = oracle.gaussian_sketch(6, c, m)
    with pytest.raises(cur.CurError) as e:
        ctx.sketch_fx(dev(G), Ad)
    assert e.value.status == cur.CUR_EINVAL
    Afull = rng.standard_normal((m, n + 5))
    Ad = dev(Afull)[:, 1:n + 1]                # stride n + 5 (even), base + 8 bytes: rejected
    with pytest.raises(cur.CurError) as e:
        ctx.sketch_fx(dev(G), Ad)
    assert e.value.status == cur.CUR_EINVAL
    Ad = dev(Afull)[:, :n]                     # stride n + 5 = 306, aligned base
    Y, _ = ctx.sketch_fx(dev(G), Ad)
    Yo = oracle.sketch_fx(oracle.quantize_q8(G), np.ascontiguousarray(Afull[:, :n]))
    np.testing.assert_array_equal(Y.cpu().numpy(), Yo)
    Afull[5, 17] = np.inf
    Y, ss = ctx.sketch_fx(dev(G), dev(Afull)[:, :n])
    Y = Y.cpu().numpy()
    assert np.all(np.isnan(Y[:, 17])) and np.all(np.isfinite(np.delete(Y, 17, axis=1)))
    assert not np.isfinite(ss)


def test_sketch_fx_repeat_is_bitwise(ctx):
    A = dev(np.random.default_rng(8).standard_normal((3000, 700)))
    G = dev(oracle.gaussian_sketch(9, 55, 3000))
    Y1, s1 = ctx.sketch_fx(G, A)
    Y2, s2 = ctx.sketch_fx(G, A)
    assert torch.equal(Y1, Y2) and s1 == s2


@pytest.mark.parametrize("seed", [0, 5])   # seeds whose oracle decisions are all clear of rounding
def test_small_workload_parity_fx(ctx, seed):
    """1000 x 800, s_i = 10^(-i/50), tol 1e-6, b = 10, c = 30 in the FP64
    tensor-core form."""
    import paper_2509_21963_gb300 as cur
    A = inputs.cfg_small(seed)
    ref = oracle.run_fx(A, 1e-6, 10, 30, seed=seed)
    got = ctx.run(dev(A), 1e-6, 10, 30, seed, sketch_mode=cur.CUR_SKETCH_F64_TC)
    _check_parity(A, got, ref, 10)
    assert got.status == 0 and got.rho <= 1e-6
    assert oracle.true_error(A, got.I, got.J, got.U) <= 2e-6


@pytest.mark.parametrize("m,n,b,c,tol", [
    (777, 1234, 7, 9, 1e-8),
    (3000, 50, 8, 8, 1e-10),
    (40, 3000, 16, 17, 1e-9),
    (2500, 900, 25, 140, 1e-7),       # c > 64: three passes of A
])
def test_shapes_parity_fx(ctx, m, n, b, c, tol):
    import paper_2509_21963_gb300 as cur
    k = min(m, n)
    A = inputs.svd_matrix(m, n, 0.8 ** np.arange(k), seed=m + n)
    ref = oracle.run_fx(A, tol, b, c, seed=9)
    got = ctx.run(dev(A), tol, b, c, 9, sketch_mode=cur.CUR_SKETCH_F64_TC)
    _check_parity(A, got, ref, b, require_full=False)


def test_exact_rank_recovery_fx(ctx):
    import paper_2509_21963_gb300 as cur
    A = inputs.exact_rank(500, 400, 37, seed=4)
    got = ctx.run(dev(A), 1e-10, 10, 30, 2, sketch_mode=cur.CUR_SKETCH_F64_TC)
    assert got.status == 0 and got.rank == 40
    assert oracle.true_error(A, got.I, got.J, got.U) < 1e-12 and got.rho < 1e-12


def test_host_entry_point_fx(ctx):
    import paper_2509_21963_gb300 as cur
    A = inputs.cfg_small(1)
    a = ctx.run(dev(A), 1e-6, 10, 30, 1, sketch_mode=cur.CUR_SKETCH_F64_TC)
    h = ctx.run_host(A, 1e-6, 10, 30, 1, sketch_mode=cur.CUR_SKETCH_F64_TC)
    assert np.array_equal(a.I, h.I) and np.array_equal(a.J, h.J)
    assert a.rho == h.rho and np.array_equal(a.U, h.U)


def test_fx_rejects_fp32(ctx):
    import paper_2509_21963_gb300 as cur
    A = dev(inputs.cfg_small(0).astype(np.float32))
    with pytest.raises(cur.CurError) as e:
        ctx.run(A, 1e-6, 10, 30, 0, sketch_mode=cur.CUR_SKETCH_F64_TC)
    assert e.value.status == cur.CUR_EINVAL


@pytest.mark.parametrize("tol,noise", [(1e-2, 1e-8), (1e-3, 1e-10)])
def test_full_size_parity_fx(ctx, tol, noise):
    """The 20000^2 FP64 workload bench.py times, in the FP64 tensor-core form:
    the sketch equals the oracle's on sampled columns bit for bit, and the
    oracle's whole run (from its own exact sketch) agrees on I and J exactly."""
    import paper_2509_21963_gb300 as cur
    m = n = 20000
    A = inputs.decay_matrix_torch(m, n, "poly2", seed=11, noise=noise, dtype=torch.float64)
    G = ctx.gaussian(0, 55, m)
    Y, _ = ctx.sketch_fx(G, A)
    got = ctx.run(A, tol, 50, 55, 0, sketch_mode=cur.CUR_SKETCH_F64_TC)
    Ah = A.cpu().numpy()
    Y = Y.cpu().numpy()
    del A
    torch.cuda.empty_cache()
    Gq = oracle.gaussian_sketch_q8(0, 55, m)
    cols = np.random.default_rng(1).choice(n, 64, replace=False)
    np.testing.assert_array_equal(Y[:, cols], oracle.sketch_fx(Gq, np.ascontiguousarray(Ah[:, cols])))
    ref = oracle.run_fx(Ah, tol, 50, 55, seed=0)
    _check_parity(Ah, got, ref, 50)
    assert got.status == 0 and got.rho <= tol
