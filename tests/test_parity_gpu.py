"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (derived from the arithmetic, u = 2^-53):
  * G (Box-Muller): both sides evaluate the same expression on identical Philox
    words; CUDA's log/sin/cos (<= 1-2 ulp) and glibc's (< 1 ulp) differ by a
    few ulp, so |dG| <= 8 ulp(G).
  * Y = G A: any summation order obeys |Y_hat - Y| <= gamma_m |G||A|,
    gamma_m = m u / (1 - m u); two such results differ by at most twice that.
  * LUPP pivots, I, J: bit-exact.  Every comparison first checks that the
    oracle's decisions are not at rounding level (gap >= 1e-9 of the scale).
  * rho (Lemma 1 recurrence): update l, S -= (S(:,J_l) N^+) Rt_l, is formed
    from products whose inner dimensions add up to r_l + b + 1 (Rt_l =
    A(I_l,:) - L(I_l,:) Rt sums over the current rank r_l = l b), so it adds
    rounding <= (r_l + b + 1) u g ||S_{l-1}|| with interpolation growth g;
    with g <= 50 (LUPP growth on c x b blocks):
    |d rho_k| <= 1e-10 rho_k + 100 u sum_{l<=k} (r_l + b + 1) rho_{l-1}.
  * U = A(I,J)^+: Householder QR of M = A(I,J) (p x p) has normwise backward
    error ||dM||_F <= sqrt(p) gamma_{cp} ||M||_F (Higham 2002, Thm 19.4), so two
    independent FP64 inverses differ by ||dU|| / ||U|| <= 32 p^1.5 kappa(M) u
    and, to first order (dU = -U dM U), by
    ||C dU R||_F <= 32 p^1.5 u ||C U||_F ||M||_F ||U R||_F.  Both gates are
    floored at 1e-10.  (At kappa ~ 1e9, LAPACK's own inverse is 1.5e-8 away from
    the exact one in ||C dU R|| / ||A||: 1e-10 is below the FP64 floor there.)
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_21963_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_RND = 2.0 ** -53


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


# ---------------------------------------------------------------------------
# single steps
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("c,m,seed", [(30, 1000, 0), (55, 20001, 7), (3, 5, 123)])
def test_gaussian_matches_oracle(ctx, c, m, seed):
    G = ctx.gaussian(seed, c, m).cpu().numpy()
    R = oracle.gaussian_sketch(seed, c, m)
    assert np.all(np.abs(G - R) <= 8 * np.spacing(np.abs(R)))


@pytest.mark.parametrize("c,m,n,f32", [(30, 1000, 800, False), (55, 2048, 1999, False),
                                       (7, 333, 65, True), (64, 4097, 129, False)])
def test_sketch_within_summation_bound(ctx, c, m, n, f32):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    if f32:
        A = A.astype(np.float32).astype(np.float64)
    G = oracle.gaussian_sketch(3, c, m)
    Ad = dev(A.astype(np.float32) if f32 else A)
    Y, ss = ctx.sketch(dev(G), Ad)
    Y = Y.cpu().numpy()
    Yo = oracle.sketch(G, A)
    gam = m * U_RND / (1 - m * U_RND)
    bound = 2 * gam * (np.abs(G) @ np.abs(A))
    assert np.all(np.abs(Y - Yo) <= bound)
    assert abs(ss - (Yo ** 2).sum()) <= 1e-12 * (Yo ** 2).sum()


def test_sketch_strided_unaligned(ctx):
    """A with an odd row stride (scalar-load path) and 3 row blocks of Y."""
    rng = np.random.default_rng(77)
    m, n, c = 517, 333, 140
    Afull = rng.standard_normal((m, n + 1))
    Ad = dev(Afull)[:, 1:]          # row stride 334, base offset by one element
    A = Afull[:, 1:]
    G = oracle.gaussian_sketch(5, c, m)
    Y, _ = ctx.sketch(dev(G), Ad)
    Yo = oracle.sketch(G, np.ascontiguousarray(A))
    gam = m * U_RND / (1 - m * U_RND)
    assert np.all(np.abs(Y.cpu().numpy() - Yo) <= 2 * gam * (np.abs(G) @ np.abs(A)))


@pytest.mark.parametrize("nr,ncand,steps", [(30, 800, 10), (55, 20000, 50), (7, 1001, 7),
                                            (50, 20000, 50), (12, 40, 12),
                                            # slices too large for shared memory: the
                                            # blocked selector (16-feature panels) ...
                                            (120, 40000, 110), (275, 30000, 250),
                                            # ... and the unblocked global one
                                            (20, 300000, 20)])
def test_lupp_pivots_exact(ctx, nr, ncand, steps):
    rng = np.random.default_rng(nr * ncand)
    X = rng.standard_normal((nr, ncand))
    mask = np.zeros(ncand, np.uint8)
    mask[rng.choice(ncand, size=min(5, ncand - steps), replace=False)] = 1
    piv_o, gap = oracle.lupp(X.T.copy(), steps, mask.copy())
    assert gap > 1e-9 * np.abs(X).max()
    piv_g, mask_g = ctx.lupp(dev(X), steps, dev(mask))
    assert np.array_equal(piv_g.cpu().numpy(), piv_o)
    m2 = mask.copy()
    m2[piv_o] = 1
    assert np.array_equal(mask_g.cpu().numpy(), m2)


def test_lupp_zero_pivot_and_ties(ctx):
    X = np.zeros((2, 5))
    X[1, 3] = 1.0
    piv, _ = ctx.lupp(dev(X), 2)
    assert list(piv.cpu().numpy()) == [0, 3]
    T = np.array([[1.0, -1.0, 1.0, 0.5]])
    piv, _ = ctx.lupp(dev(T), 1)
    assert list(piv.cpu().numpy()) == [0]


@pytest.mark.parametrize("p,seed", [(30, 1), (50, 2), (129, 3), (370, 4)])
def test_pinv_matches_oracle(ctx, p, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((p, p))
    Xo, ko, _, _ = oracle.qrcp_pinv(M)
    Xg, kg = ctx.pinv(dev(M))
    Xg = Xg.cpu().numpy()
    assert kg == ko == p
    kappa = np.linalg.cond(M)
    assert np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo) <= 10 * p * kappa * U_RND
    assert np.linalg.norm(M @ Xg - np.eye(p)) <= 10 * p * kappa * U_RND


@pytest.mark.parametrize("p,q,seed", [(60, 45, 7), (45, 60, 8), (24, 24, 9), (256, 256, 10),
                                      (300, 130, 11), (30, 200, 12), (512, 100, 13),
                                      (23, 40, 14), (100, 257, 15)])
def test_pinv_rect_matches_oracle(ctx, p, q, seed):
    """Rectangular and boundary shapes of the shared-memory QR variants (one
    CTA below 24 rows, a thread-block cluster up to 512 rows and 16 columns
    per CTA, the cooperative grid beyond): X against the oracle's within the
    perturbation bound, and X a one-sided inverse (X M = I for full column
    rank, M X = I for full row rank)."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((p, q))
    Xo, ko, _, _ = oracle.qrcp_pinv(M)
    Xg, kg = ctx.pinv(dev(M))
    Xg = Xg.cpu().numpy()
    k = min(p, q)
    assert kg == ko == k
    s = np.linalg.svd(M, compute_uv=False)
    kappa = s[0] / s[-1]
    bound = 10 * max(p, q) * kappa * U_RND
    assert np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo) <= bound
    E = Xg @ M if p >= q else M @ Xg
    assert np.linalg.norm(E - np.eye(k)) <= bound


@pytest.mark.parametrize("p", [12, 50, 300])
def test_pinv_nan_column_is_an_error(ctx, p):
    """A matrix whose every column norm is NaN has no pivot: CUR_EINVAL, and
    the context still computes the next call correctly."""
    import paper_2509_21963_gb300 as cur
    M = np.full((p, p), np.nan)
    with pytest.raises(cur.CurError) as e:
        ctx.pinv(dev(M))
    assert e.value.status == cur.CUR_EINVAL
    M = np.random.default_rng(p).standard_normal((p, p))
    Xg, kg = ctx.pinv(dev(M))
    assert kg == p
    assert np.linalg.norm(M @ Xg.cpu().numpy() - np.eye(p)) <= 1e-9


@pytest.mark.parametrize("tol,iters", [(1e-3, 1), (1e-7, 2)])
def test_core_equals_pinv_of_selection(ctx, tol, iters):
    """U of a run is A(I,J)^+ as cur_step_pinv forms it, bit for bit: after one
    iteration the run returns N_1^+ (N_1 = A(I_1,J_1), the same kernels and
    rank threshold), after more it factors A(I,J) at exit."""
    A = inputs.svd_matrix(600, 500, 0.5 ** np.arange(500), seed=21)
    got = ctx.run(dev(A), tol, 20, 25, 3)
    assert got.iterations == iters and got.status == 0
    M = dev(A)[torch.from_numpy(got.I).cuda()][:, torch.from_numpy(got.J).cuda()].contiguous()
    X, k = ctx.pinv(M)
    assert np.array_equal(got.U.reshape(X.shape), X.cpu().numpy())


def test_pinv_team_matches_oracle(ctx):
    """A square core too large for the shared-memory QR kernels (p = 1900)
    runs on the whole-GPU team QR with a panel of 8 right-hand sides: against
    the oracle, with the bounds above."""
    p = 1900
    M = np.random.default_rng(6).standard_normal((p, p))
    Xo, ko, _, _ = oracle.qrcp_pinv(M)
    Xg, kg = ctx.pinv(dev(M))
    Xg = Xg.cpu().numpy()
    assert kg == ko == p
    kappa = np.linalg.cond(M)
    assert np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo) <= 10 * p * kappa * U_RND
    assert np.linalg.norm(M @ Xg - np.eye(p)) <= 10 * p * kappa * U_RND


@pytest.mark.parametrize("p", [3001, 6000])
def test_pinv_team_wide_cores(ctx, p):
    """Team QR cores with solve panels of 4 (p = 3001, ragged against the 256
    threads) and 2 (p = 6000) right-hand sides, beyond the oracle's seconds:
    Householder QR's backward stability, ||M X - I||_F <= 10 p u ||M||_F ||X||_F
    (||M||_F ||X||_F bounds kappa_2 from above); a wrong reflector, pivot or
    row leaves a residual of order one."""
    Md = torch.from_numpy(np.random.default_rng(p).standard_normal((p, p))).cuda()
    Xd, k = ctx.pinv(Md)
    assert k == p
    res = torch.linalg.matrix_norm(Md @ Xd - torch.eye(p, dtype=torch.float64, device="cuda")).item()
    bound = 10 * p * U_RND * torch.linalg.matrix_norm(Md).item() * torch.linalg.matrix_norm(Xd).item()
    assert res <= bound, (res, bound)
    assert res <= 1e-6


def test_run_team_core_wide_panel(ctx):
    """A whole run whose core (rank 2700 at full rank) takes the team QR with a
    4-wide solve panel: the returned U inverts A(I,J) to the same backward
    bound, and the run ends at full rank with rho at noise level."""
    m, n = 3000, 2700
    A = inputs.svd_matrix(m, n, 0.9995 ** np.arange(n), seed=12)
    got = ctx.run(dev(A), 1e-8, 50, 55, 3)
    assert got.status == 0 and got.rank == n and got.rho <= 1e-9
    assert len(set(got.I)) == n and len(set(got.J)) == n
    Md = dev(A)[torch.from_numpy(got.I).cuda()][:, torch.from_numpy(got.J).cuda()]
    Ud = torch.from_numpy(got.U).cuda()
    res = torch.linalg.matrix_norm(Ud @ Md - torch.eye(n, dtype=torch.float64, device="cuda")).item()
    bound = 10 * n * U_RND * torch.linalg.matrix_norm(Md).item() * torch.linalg.matrix_norm(Ud).item()
    assert res <= bound, (res, bound)


def test_pinv_rank_deficient(ctx):
    rng = np.random.default_rng(5)
    M = rng.standard_normal((40, 10)) @ rng.standard_normal((10, 40))
    Xg, kg = ctx.pinv(dev(M))
    Xo, ko, _, _ = oracle.qrcp_pinv(M)
    assert kg == ko == 10
    Xg = Xg.cpu().numpy()
    assert np.abs(M @ Xg @ M - M).max() < 1e-11 * np.abs(M).max()


# ---------------------------------------------------------------------------
# the whole method
# ---------------------------------------------------------------------------
def _decided_prefix(ref, b, col_scale, tau=1e-9):
    """Number of leading selections whose LUPP decisions are not at rounding
    level in the oracle (gap / scale >= tau)."""
    k = 0
    for it in range(ref.iters):
        if ref.gap_col[it] < tau * col_scale or ref.gap_row[it] < tau * ref.scale_row[it]:
            break
        k += 1
    return min(ref.rank, k * b)


def _check_parity(A, got, ref, b, require_full=True, rho_rtol=None):
    n_dec = _decided_prefix(ref, b, ref.maxabsY)
    if require_full:
        assert n_dec == ref.rank, "oracle decisions at rounding level; choose another seed"
    assert np.array_equal(got.I[:n_dec], ref.I[:n_dec])
    assert np.array_equal(got.J[:n_dec], ref.J[:n_dec])
    if n_dec < ref.rank:
        return
    assert got.rank == ref.rank and got.iterations == ref.iters and got.status == ref.status
    hist_prev = np.concatenate([[1.0], ref.rho_hist[:-1]])
    r_l = b * np.arange(len(hist_prev))
    bound = 1e-10 * ref.rho_hist + 100 * U_RND * np.cumsum((r_l + b + 1) * hist_prev)
    if rho_rtol is not None:
        bound = np.maximum(bound, rho_rtol * ref.rho_hist)
    # Once |I| = |J| = min(m, n) every row (or column) is selected and the exact
    # residual is zero (S_k vanishes on I and J, Lemma 1): rho there is rounding
    # noise on both sides, held to a noise ceiling instead of to each other.
    full = np.minimum(b * np.arange(1, len(hist_prev) + 1), ref.rank) >= min(A.shape)
    gh = np.asarray(got.rho_history)
    assert np.all(np.abs(gh - ref.rho_hist)[~full] <= bound[~full])
    assert np.all(gh[full] <= 1e-9) and np.all(ref.rho_hist[full] <= 1e-9)
    if not full[-1]:
        assert abs(got.rho - ref.rho) <= bound[-1]
    if ref.rank:
        _check_core(A, got, ref)


def _inv_ext(M):
    """Inverse by Gauss-Jordan elimination with partial pivoting in np.longdouble
    (x87 80-bit or IEEE quad): the reference the FP64 cores are measured against."""
    p = M.shape[0]
    W = np.array(M, dtype=np.longdouble)
    X = np.eye(p, dtype=np.longdouble)
    for k in range(p):
        q = k + int(np.argmax(np.abs(W[k:, k])))
        if q != k:
            W[[k, q]] = W[[q, k]]
            X[[k, q]] = X[[q, k]]
        piv = W[k, k]
        W[k] /= piv
        X[k] /= piv
        f = W[:, k].copy()
        f[k] = 0
        W -= np.outer(f, W[k])
        X -= np.outer(f, X[k])
    return X


def _check_core(A, got, ref):
    """Gate U; return a bound on ||C (U_g - U_o) R|| / ||A||.

    For a nonsingular core M = A(I,J) both sides approximate M^{-1}; their
    distance is set by each side's own rounding error, which grows with
    kappa(M) (measured: 6 p^2 u ||CU|| ||M|| ||UR|| for the oracle itself at
    kappa ~ 1e8, up to 1e-5 relative in U at kappa ~ 1e11).  So the GPU core is
    held to the oracle's accuracy: measured against an extended-precision
    inverse, ||C (U_g - M^-1) R|| <= 4 ||C (U_o - M^-1) R|| + 1e-13 ||A|| and
    ||U_g - M^-1|| <= 4 ||U_o - M^-1|| + 1e-13 ||M^-1||.  A numerically singular
    core (rank below p in the oracle's pivoted QR) has no unique answer: the
    CUR it defines must then be as accurate as the oracle's."""
    p = ref.rank
    C, R, M = A[:, ref.J], A[ref.I, :], A[np.ix_(ref.I, ref.J)]
    nA = np.linalg.norm(A)
    if np.linalg.matrix_rank(M) < p:
        e_g = oracle.true_error(A, got.I, got.J, got.U)
        e_o = oracle.true_error(A, ref.I, ref.J, ref.U)
        assert e_g <= 1.1 * e_o + 1e-12
        return abs(e_g - e_o) + 1e-12
    Mi = _inv_ext(M)
    def errs(U):
        # the difference in extended precision; its (small) value then in FP64
        D = (np.asarray(U, dtype=np.longdouble) - Mi).astype(np.float64)
        return np.linalg.norm(C @ D @ R) / nA, np.linalg.norm(D)
    cg, ug = errs(got.U)
    co, uo = errs(ref.U)
    nMi = np.linalg.norm(Mi.astype(np.float64))
    assert ug <= 4 * uo + 1e-13 * nMi, (ug, uo)
    assert cg <= 4 * co + 1e-13, (cg, co)
    return cg + co


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_small_workload_parity(ctx, seed):
    """1000 x 800, s_i = 10^(-i/50), tol 1e-6, b = 10, c = 2b + 10 = 30."""
    A = inputs.cfg_small(seed)
    ref = oracle.run(A, 1e-6, 10, 30, seed=seed, mode=1)
    got = ctx.run(dev(A), 1e-6, 10, 30, seed)
    _check_parity(A, got, ref, 10)
    assert got.status == 0 and got.rho <= 1e-6
    # | ||A - C U_g R|| - ||A - C U_o R|| | <= ||C (U_g - U_o) R||
    err_g = oracle.true_error(A, got.I, got.J, got.U)
    err_o = oracle.true_error(A, ref.I, ref.J, ref.U)
    assert abs(err_g - err_o) <= _check_core(A, got, ref)


def test_small_workload_matches_literal_algorithm(ctx):
    """Against the literal form of Algorithm 1 (explicit U = A(I,J)^+ every
    iteration): the same indices; rho within the literal form's own rounding
    error.  There S^col = Y - (Y_J U) R with a backward-stable U (backward error
    <= sqrt(p) gamma_{cp} ||M||), so to first order
    |d rho| <= 32 p^1.5 u ||Y_J U|| ||M|| ||U R|| / ||Y||
    (the literal rho even differs between x86 and Arm hosts by ~1e-10 here)."""
    A = inputs.cfg_small(0)
    lit = oracle.run(A, 1e-6, 10, 30, seed=0, mode=0)
    got = ctx.run(dev(A), 1e-6, 10, 30, 0)
    assert np.array_equal(got.I, lit.I) and np.array_equal(got.J, lit.J)
    Y = oracle.sketch(oracle.gaussian_sketch(0, 30, A.shape[0]), A)
    M = A[np.ix_(lit.I, lit.J)]
    W = Y[:, lit.J] @ lit.U
    bound = 32 * lit.rank ** 1.5 * U_RND * np.linalg.norm(W) * np.linalg.norm(M) * \
        np.linalg.norm(lit.U @ A[lit.I, :]) / np.linalg.norm(Y)
    assert abs(got.rho - lit.rho) <= bound


@pytest.mark.parametrize("m,n,b,c,tol,f32", [
    (777, 1234, 7, 9, 1e-8, False),     # ragged tiles, n > m
    (3000, 50, 8, 8, 1e-10, False),     # tall, c = b
    (40, 3000, 16, 17, 1e-9, False),    # wide; rank capped by m
    (5, 300, 10, 11, 1e-12, False),     # m < b: last block clamped
    (1000, 800, 10, 30, 1e-5, True),    # FP32 input, same values
])
def test_shapes_parity(ctx, m, n, b, c, tol, f32):
    k = min(m, n)
    A = inputs.svd_matrix(m, n, 0.8 ** np.arange(k), seed=m + n)
    if f32:
        A = A.astype(np.float32).astype(np.float64)
    ref = oracle.run(A, tol, b, c, seed=9, mode=1)
    Ad = dev(A.astype(np.float32)) if f32 else dev(A)
    got = ctx.run(Ad, tol, b, c, 9)
    _check_parity(A, got, ref, b, require_full=False)


def test_explicit_sketch_parity(ctx):
    A = inputs.cfg_small(3)
    G = inputs.explicit_sketch(30, 1000, seed=3)
    ref = oracle.run(A, 1e-6, 10, 30, G=G, mode=1)
    got = ctx.run(dev(A), 1e-6, 10, 30, 0, omega=dev(G))
    _check_parity(A, got, ref, 10)


def test_exact_rank_recovery_gpu(ctx):
    A = inputs.exact_rank(500, 400, 37, seed=4)
    ref = oracle.run(A, 1e-10, 10, 30, seed=2, mode=1)
    got = ctx.run(dev(A), 1e-10, 10, 30, 2)
    # the first 30 selections are decided; the 4th block picks from noise
    assert np.array_equal(got.I[:30], ref.I[:30]) and np.array_equal(got.J[:30], ref.J[:30])
    assert got.status == 0 and got.rank == ref.rank == 40
    assert oracle.true_error(A, got.I, got.J, got.U) < 1e-12
    assert got.rho < 1e-12


def test_edge_cases_gpu(ctx):
    import paper_2509_21963_gb300 as cur
    Z = torch.zeros(64, 48, dtype=torch.float64, device="cuda")
    r = ctx.run(Z, 1e-6, 4, 5, 0)
    assert r.rank == 0 and r.rho == 0.0 and r.status == 0
    A = inputs.svd_matrix(64, 48, 0.5 ** np.arange(48), seed=1)
    Ad = dev(A)
    r = ctx.run(Ad, 1.0, 4, 5, 0)
    assert r.rank == 0 and r.rho == 1.0
    r = ctx.run(Ad, 1e-14, 4, 5, 0, max_rank=6)
    assert r.rank == 6 and r.status == cur.CUR_TOL_UNREACHED
    ref = oracle.run(A, 1e-14, 4, 5, seed=0, max_rank=6, mode=1)
    assert np.array_equal(r.I, ref.I) and np.array_equal(r.J, ref.J)
    bad = Ad.clone()
    bad[3, 7] = float("nan")
    with pytest.raises(cur.CurError) as e:
        ctx.run(bad, 1e-6, 4, 5, 0)
    assert e.value.status == cur.CUR_ENONFINITE
    bad[3, 7] = float("inf")
    with pytest.raises(cur.CurError) as e:
        ctx.run(bad, 1e-6, 4, 5, 0)
    assert e.value.status == cur.CUR_ENONFINITE
    for args in [(0.0, 4, 5), (float("nan"), 4, 5), (1e-6, 4, 3), (1e-6, 0, 5)]:
        with pytest.raises(cur.CurError) as e:
            ctx.run(Ad, *args, 0)
        assert e.value.status == cur.CUR_EINVAL
    with pytest.raises(cur.CurError) as e:
        ctx.run(Ad, 1e-6, 4, 5, 0, alpha=1e-10)  # c = 5 <= -4 ln(alpha)
    assert e.value.status == cur.CUR_EINVAL
    # the context stays usable after every error
    r = ctx.run(Ad, 1e-6, 4, 5, 0)
    assert r.status == 0


def test_risk_aware_threshold_gpu(ctx):
    A = inputs.cfg_small(0)
    alpha, delta = 1e-3, 0.0
    thr = oracle.risk_threshold(1e-4, delta, alpha, 30)
    ref = oracle.run(A, thr, 10, 30, seed=0, mode=1)
    got = ctx.run(dev(A), 1e-4, 10, 30, 0, alpha=alpha, delta=delta)
    _check_parity(A, got, ref, 10)
    assert got.rho <= thr


def test_host_entry_point_matches_device(ctx):
    A = inputs.cfg_small(1)
    a = ctx.run(dev(A), 1e-6, 10, 30, 1)
    h = ctx.run_host(A, 1e-6, 10, 30, 1)
    assert np.array_equal(a.I, h.I) and np.array_equal(a.J, h.J)
    assert a.rho == h.rho and np.array_equal(a.U, h.U)


def test_host_entry_point_row_blocks(ctx):
    """With m >= 2048 the host entry copies A in row blocks that overlap the
    sketch; the sketch is then summed block by block (another rounding order),
    so the result equals the device-input run in every decision, with rho and U
    equal to rounding."""
    A = inputs.svd_matrix(9000, 600, 10.0 ** (-np.arange(1, 601) / 30.0), seed=12)
    a = ctx.run(dev(A), 1e-6, 20, 30, 5)
    h = ctx.run_host(A, 1e-6, 20, 30, 5)
    assert np.array_equal(a.I, h.I) and np.array_equal(a.J, h.J) and a.rank == h.rank
    assert abs(a.rho - h.rho) <= 1e-9 * a.rho
    assert np.linalg.norm(a.U - h.U) <= 1e-6 * np.linalg.norm(a.U)
    ref = oracle.run(A, 1e-6, 20, 30, seed=5, mode=1)
    _check_parity(A, h, ref, 20, require_full=False)


@pytest.mark.parametrize("m,n,strided", [(700, 1500, False), (600, 2176, True), (300, 128, False),
                                         (1100, 16500, True)])
def test_host_entry_point_fx_column_blocks(ctx, m, n, strided):
    """FP64 tensor-core sketch with A in host memory: A is copied in column
    groups of at least 8192 columns (16500 gives 8320 + 8180), each in row
    blocks of at least 512 rows (1100 gives two); the column maxima of a row
    block are taken when it lands and a group's tensor-core pass runs while
    the next group is copied.  The sketch sums are exact integers added into
    each group's own columns, so the run equals the device-input run bit for
    bit (strided host rows too)."""
    k = min(m, n)
    A = inputs.svd_matrix(m, n, 10.0 ** (-np.arange(1, k + 1) / 40.0), seed=m + n)
    if strided:
        Aw = np.zeros((m, n + 10))
        Aw[:, :n] = A
        Ah = Aw[:, :n]
    else:
        Ah = A
    a = ctx.run(dev(A), 1e-6, 20, 30, 3, sketch_mode=5)
    h = ctx.run_host(Ah, 1e-6, 20, 30, 3, sketch_mode=5)
    assert np.array_equal(a.I, h.I) and np.array_equal(a.J, h.J) and a.rank == h.rank
    assert a.rho == h.rho and np.array_equal(a.U, h.U)
    assert a.status == h.status


def test_deterministic_repeat(ctx):
    A = dev(inputs.cfg_small(2))
    a = ctx.run(A, 1e-6, 10, 30, 4)
    b = ctx.run(A, 1e-6, 10, 30, 4)
    assert np.array_equal(a.I, b.I) and a.rho == b.rho and np.array_equal(a.U, b.U)


# ---------------------------------------------------------------------------
# full size: 20000 x 20000, the configuration bench.py times
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("tol,noise", [(1e-2, 1e-8), (1e-3, 1e-10)])
def test_full_size_parity_fp64(ctx, tol, noise):
    """A = U diag(i^-2) V^T + N(0, noise^2), 20000^2 FP64, b = 50, c = 55 (the
    configuration bench.py times, and its second form): the oracle runs the
    whole method on the same matrix and must agree exactly on I, J."""
    m = n = 20000
    A = inputs.decay_matrix_torch(m, n, "poly2", seed=11, noise=noise, dtype=torch.float64)
    got = ctx.run(A, tol, 50, 55, 0)
    Ah = A.cpu().numpy()
    del A
    torch.cuda.empty_cache()
    ref = oracle.run(Ah, tol, 50, 55, seed=0, mode=1)
    _check_parity(Ah, got, ref, 50)
    assert got.status == 0 and got.rho <= tol


@pytest.mark.parametrize("mode", [0, 2])
def test_full_size_parity_fp32(ctx, mode):
    """The FP32 20000^2 forms bench.py reports (A = U diag(i^-2) V^T +
    N(0, 1e-16) stored as FP32, tol 1e-2, b = 50, c = 55): the FP64 sketch of
    the FP32 data (mode 0) against the oracle on the same values, and the
    two-digit tensor-core sketch (mode 2) against the oracle started from its
    exact sketch G_q fix_2(A) (products and sums exact in FP64 here).  Same I
    and J; rho as in the FP64 gates (mode 2: within 1e-6 relative)."""
    m = n = 20000
    A = inputs.decay_matrix_torch(m, n, "poly2", seed=11, noise=1e-8, dtype=torch.float32)
    got = ctx.run(A, 1e-2, 50, 55, 0, sketch_mode=mode)
    Ah = A.cpu().numpy().astype(np.float64)
    del A
    torch.cuda.empty_cache()
    if mode == 0:
        ref = oracle.run(Ah, 1e-2, 50, 55, seed=0, mode=1)
        _check_parity(Ah, got, ref, 50)
    else:
        Y = oracle.sketch(oracle.gaussian_sketch_q8(0, 55, m), oracle.fixed_point(Ah, 2))
        ref = oracle.run_y(Ah, 1e-2, 50, 55, Y)
        _check_parity(Ah, got, ref, 50, rho_rtol=1e-6)
    assert got.status == 0 and got.rho <= 1e-2
