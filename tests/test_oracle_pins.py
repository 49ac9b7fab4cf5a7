"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks one oracle function against what the paper prints, a closed
form, an invariant, a library routine the oracle does not use, or brute force,
chosen so that a dropped term, a wrong sign/index or a transposed operand in
the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
from paper_2509_21963_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


# --------------------------------------------------------------------------
# Philox4x64-10 (Salmon et al. SC'11) against numpy's independent Philox.
# numpy increments the 256-bit counter before each block, so the block at
# counter c is numpy's first output when started from c - 1.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ctr,key", [
    ([5, 3, 0, 0], [123, 0x43555200]),
    ([0, 7, 0, 0], [0, 1]),
    ([2**64 - 1, 2**64 - 1, 5, 9], [2**64 - 1, 3]),
    ([17, 2**40 + 3, 2**63, 1], [0xDEADBEEF, 2**64 - 2]),
])
def test_philox_matches_numpy(ctr, key):
    ours = oracle.philox4x64_10(np.array(ctr, dtype=np.uint64), np.array(key, dtype=np.uint64))
    cint = (sum(int(c) << (64 * i) for i, c in enumerate(ctr)) - 1) % (1 << 256)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=cint)
    ref = bg.random_raw(4)
    assert np.array_equal(ours, ref)


def test_gaussian_sketch_is_standard_normal():
    G = oracle.gaussian_sketch(11, 16, 40000)
    z = G.ravel()
    n = z.size
    assert abs(z.mean()) < 5.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(scipy.stats.kurtosis(z, fisher=False) - 3.0) < 5.0 * math.sqrt(24.0 / n)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # rows are independent streams: sample correlation of two rows ~ N(0, 1/m)
    C = np.corrcoef(G)
    off = C[~np.eye(16, dtype=bool)]
    assert np.abs(off).max() < 6.0 / math.sqrt(40000)
    # deterministic in the seed, different across seeds, ragged tail handled
    assert np.array_equal(G[:, :39998], oracle.gaussian_sketch(11, 16, 39998))
    assert not np.array_equal(G, oracle.gaussian_sketch(12, 16, 40000))


def test_sketch_matches_numpy_matmul():
    rng = np.random.default_rng(3)
    G = rng.standard_normal((13, 57))
    A = rng.standard_normal((57, 41))
    Y = oracle.sketch(G, A)
    np.testing.assert_allclose(Y, G @ A, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# LUPP selector against LAPACK getrf (scipy.linalg.lu).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p,q", [(40, 7), (200, 30), (9, 9)])
def test_lupp_pivots_match_lapack(p, q):
    rng = np.random.default_rng(p * 31 + q)
    M = rng.standard_normal((p, q))
    P, L, U = scipy.linalg.lu(M)
    perm = np.argmax(P, axis=0)  # (P^T M)[i] = M[perm[i]]
    piv, gap = oracle.lupp(M, q)
    assert np.array_equal(piv, perm[:q])
    assert gap > 0
    # fewer steps = the first pivots (a later step cannot change earlier ones)
    piv3, _ = oracle.lupp(M, 3)
    assert np.array_equal(piv3, perm[:3])


def test_lupp_exclusion_is_lu_on_eligible_rows():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((50, 6))
    ex = np.zeros(50, np.uint8)
    ex[[3, 17, 20, 41]] = 1
    keep = np.flatnonzero(ex == 0)
    piv, _ = oracle.lupp(M, 6, ex.copy())
    P, _, _ = scipy.linalg.lu(M[keep])
    assert np.array_equal(piv, keep[np.argmax(P, axis=0)[:6]])
    # the chosen rows are marked as excluded for later calls
    ex2 = ex.copy()
    oracle.lupp(M, 6, ex2)
    assert set(np.flatnonzero(ex2 != ex)) == set(piv)


def test_lupp_zero_column_and_ties():
    M = np.zeros((5, 2))
    M[3, 1] = 1.0
    piv, _ = oracle.lupp(M, 2)
    assert list(piv) == [0, 3]  # zero pivot column -> smallest eligible index
    T = np.array([[1.0], [-1.0], [1.0]])
    assert list(oracle.lupp(T, 1)[0]) == [0]  # tie -> smallest index


# --------------------------------------------------------------------------
# Pivoted-QR generalised inverse.
# --------------------------------------------------------------------------
def test_qrcp_pinv_square_is_inverse():
    rng = np.random.default_rng(7)
    M = rng.standard_normal((30, 30))
    X, k, perm, rdiag = oracle.qrcp_pinv(M)
    assert k == 30
    np.testing.assert_allclose(X, np.linalg.inv(M), rtol=0, atol=1e-10 * np.abs(np.linalg.inv(M)).max())
    # Businger-Golub pivot order equals LAPACK geqp3 on generic data
    _, _, p_ref = scipy.linalg.qr(M, pivoting=True)
    assert np.array_equal(perm, p_ref)
    # |R| diagonal non-increasing (column pivoting invariant)
    assert np.all(np.diff(np.abs(rdiag)) <= 1e-12)


def test_qrcp_pinv_tall_is_moore_penrose():
    rng = np.random.default_rng(8)
    M = rng.standard_normal((25, 9))
    X, k, _, _ = oracle.qrcp_pinv(M)
    assert k == 9
    np.testing.assert_allclose(X, np.linalg.pinv(M), rtol=0, atol=1e-12)


def test_qrcp_pinv_rank_deficient_is_generalised_inverse():
    rng = np.random.default_rng(9)
    M = rng.standard_normal((12, 4)) @ rng.standard_normal((4, 12))
    X, k, _, _ = oracle.qrcp_pinv(M)
    assert k == 4
    np.testing.assert_allclose(M @ X @ M, M, rtol=0, atol=1e-12 * np.abs(M).max())
    np.testing.assert_allclose(X @ M @ X, X, rtol=0, atol=1e-10 * np.abs(X).max())


# --------------------------------------------------------------------------
# The whole method.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("rank", [5, 25, 37])
def test_exact_rank_recovery(mode, rank):
    """Once |J| >= rank(A), the CUR reproduces A to near machine precision
    (Sec. 5.1 reports 9e-14 on an exactly low-rank matrix)."""
    g = _golden("low_rank_accuracy.txt")["median_relative_error"]
    A = inputs.exact_rank(300, 240, rank, seed=rank)
    res = oracle.run(A, 1e-10, 10, 30, seed=1, mode=mode)
    assert res.status == 0
    assert res.rank >= rank and res.rank <= rank + 10
    err = oracle.true_error(A, res.I, res.J, res.U)
    assert err < 100 * g
    assert res.rho < 100 * g


def _example1():
    """Concrete instance of Example 1 satisfying all its stated relations."""
    v2 = np.array([2.0, 3.0, 1.0]) / math.sqrt(14.0)  # v2(2) > v2(1) > v2(3) > 0
    P = scipy.linalg.null_space(v2[None, :])           # basis of v2^perp
    p, q = P[:, 0], P[:, 1]
    th = math.atan2(q[1] - p[1], q[1] + p[1])           # v1(2) = v3(2)
    v1 = math.cos(th) * p + math.sin(th) * q
    v3 = -math.sin(th) * p + math.cos(th) * q
    if v1[1] < 0:
        v1, v3 = -v1, -v3
    assert abs(v1[1] - v3[1]) < 1e-14 and v1[1] > 0
    c1, c2, c3, d2, d3 = 3.0, 2.0, 1.0, 2.0, 1.0
    A = np.column_stack([c1 * v1, c2 * v2, c3 * v3])
    g = d2 * v2 + d3 * v3
    return A, g, (v1, v2, v3), (c1, c2, c3, d2, d3)


@pytest.mark.parametrize("mode", [0, 1])
def test_example1_self_correction(mode):
    gold = _golden("example1.txt")
    A, g, (v1, v2, v3), (c1, c2, c3, d2, d3) = _example1()
    res = oracle.run(A, 1e-300, 1, 1, G=g[None, :], max_rank=2, mode=mode)
    assert res.J[0] == gold["columns_iteration1"] - 1
    assert res.I[0] == gold["rows_iteration1"] - 1
    assert res.J[1] == gold["columns_iteration2"] - 1
    # sketched residual after iteration 1 equals the closed form of the example
    one = oracle.run(A, 1e-300, 1, 1, G=g[None, :], max_rank=1, mode=mode, want_S=True)
    expect = np.array([-c1 * d2 * v1[1] / v2[1], 0.0, c3 * d3 - c3 * d2 * v3[1] / v2[1]])
    np.testing.assert_allclose(one.S_final[0], expect, rtol=0, atol=1e-14)


def test_dependent_selection_nonzero_core():
    """Sec. 3.2 example: with dependent (columns-then-rows) selection the
    rank-1 core A(I,J) is never 0, whichever sketch is drawn."""
    nn, eta = 16, 0.05
    A = np.zeros((2, nn + 1))
    A[0, 1:] = 1.0 / math.sqrt(nn)
    A[1, 0] = 1.0 / math.sqrt(nn) + eta
    for seed in range(40):
        res = oracle.run(A, 1e-300, 1, 1, seed=seed, max_rank=1)
        core = A[res.I[0], res.J[0]]
        assert core != 0.0
        assert core in (1.0 / math.sqrt(nn), 1.0 / math.sqrt(nn) + eta)


def test_risk_threshold_worked_value():
    g = _golden("risk_threshold.txt")
    thr = oracle.risk_threshold(1.0, g["delta"], g["alpha"], g["c"])
    assert round(1.0 / thr, 2) == g["divisor"]
    assert oracle.risk_threshold(1.0, 0.0, 1e-10, 90) == -1.0  # c <= -4 ln(alpha)


def _cur(A, I, J, thr=-1.0):
    X, _, _, _ = oracle.qrcp_pinv(A[np.ix_(I, J)], thr)
    return A[:, J] @ X @ A[I, :]


def test_lemma1_recurrence():
    """Lemma 1: A_{I u I+, J u J+} = A_{I,J} + S_{I+,J+}, S = A - A_{I,J}."""
    rng = np.random.default_rng(21)
    A = rng.standard_normal((20, 18))
    I, J, Ip, Jp = [1, 7, 4], [0, 9, 3], [12, 2], [5, 16]
    S = A - _cur(A, I, J)
    lhs = _cur(A, I + Ip, J + Jp)
    rhs = _cur(A, I, J) + _cur(S, Ip, Jp)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-11)


@pytest.mark.parametrize("mode", [0, 1])
def test_interpolation_residual_vanishes_on_selection(mode):
    """Sec. 3.2.2: S(I,:) = 0 and S(:,J) = 0 for a nonsingular core."""
    A = inputs.svd_matrix(120, 90, 0.8 ** np.arange(90), seed=4)
    res = oracle.run(A, 1e-3, 8, 9, seed=2, mode=mode)
    S = A - A[:, res.J] @ res.U @ A[res.I, :]
    scale = np.abs(A).max()
    assert np.abs(S[res.I, :]).max() < 1e-10 * scale
    assert np.abs(S[:, res.J]).max() < 1e-10 * scale


def test_bruteforce_tiny_osinsky_bound():
    """Theorem 2 (Osinsky): some (I, J) with |I| = |J| = k has CUR error at most
    (k+1) times the rank-k SVD tail; the oracle's CUR can be no better than the
    brute-force optimum."""
    rng = np.random.default_rng(13)
    for trial in range(6):
        m, n, k = 6, 5, 1 + trial % 2
        A = rng.standard_normal((m, n)) @ np.diag(0.5 ** np.arange(n))
        s = np.linalg.svd(A, compute_uv=False)
        tail = math.sqrt((s[k:] ** 2).sum())
        best = min(np.linalg.norm(A - _cur(A, list(I), list(J)))
                   for I in itertools.combinations(range(m), k)
                   for J in itertools.combinations(range(n), k))
        assert best <= (k + 1) * tail * (1 + 1e-12)
        res = oracle.run(A, 1e-300, k, k, seed=trial, max_rank=k)
        err = np.linalg.norm(A - A[:, res.J] @ res.U @ A[res.I, :])
        assert err >= best * (1 - 1e-12)


def test_naive_loop_selects_the_same_indices():
    """Sec. 3.1: recycling G A (Algorithm 1) equals re-sketching the full
    residual every iteration, by linearity G (A - CUR) = GA - (GC) U R."""
    A = inputs.svd_matrix(60, 50, 0.7 ** np.arange(50), seed=6)
    G = inputs.explicit_sketch(7, 60, seed=6)
    rec = oracle.run(A, 1e-6, 6, 7, G=G, mode=0)
    nai = oracle.run_naive(A, 1e-6, 6, 7, G=G)
    assert np.array_equal(rec.I, nai.I) and np.array_equal(rec.J, nai.J)
    # rho is relative to ||G A||: the two orders of evaluation (G (A - CUR) vs
    # GA - (GC) U R) differ by rounding of the explicit U, ~kappa(A(I,J)) u.
    np.testing.assert_allclose(rec.rho_hist, nai.rho_hist, rtol=1e-6, atol=1e-10)


def test_estimator_distortion_gratton_bound():
    """Theorem 3.1 of Gratton & Titley-Peloquin (Sec. 3.3): with c Gaussian
    rows, P[||G S||_F <= ||S||_F sqrt(c) / tau] <= exp(-c (tau^2-1)^2 / (4 tau^4)).
    The oracle's sketched residual at the first iteration must respect it."""
    A = inputs.svd_matrix(80, 70, 0.85 ** np.arange(70), seed=8)
    c, b, tau = 10, 5, 1.5
    bound = math.exp(-c * (tau ** 2 - 1) ** 2 / (4 * tau ** 4))
    fails, runs = 0, 300
    for seed in range(runs):
        res = oracle.run(A, 1e-300, b, c, seed=seed, max_rank=b, want_S=True)
        S = A - A[:, res.J] @ res.U @ A[res.I, :]
        ratio = np.linalg.norm(res.S_final) / (math.sqrt(c) * np.linalg.norm(S))
        fails += ratio <= 1.0 / tau
    freq = fails / runs
    assert freq <= bound + 3 * math.sqrt(bound * (1 - bound) / runs)


@pytest.mark.parametrize("seed", [0, 1])
def test_small_workload_estimate_tracks_truth_and_decreases(seed):
    """1000 x 800, s_i = 10^(-i/50), tol 1e-6, b = 10, c = 30: the estimate
    agrees with the true error within the sketch distortion and decreases
    monotonically on this decaying spectrum."""
    A = inputs.cfg_small(seed)
    res = oracle.run(A, 1e-6, 10, 30, seed=seed, mode=1)
    assert res.status == 0 and res.rho <= 1e-6
    assert 300 <= res.rank <= 400
    err = oracle.true_error(A, res.I, res.J, res.U)
    assert 0.5 < err / res.rho < 2.0
    assert np.all(np.diff(res.rho_hist) < 0)


def test_lemma_mode_matches_extended_precision():
    """The Lemma 1 residual recurrence reproduces the sketched residual of the
    final (I, J) computed in extended precision (x87 long double with
    iterative refinement), to within 1e-7 relative at rho ~ 1e-6."""
    if np.finfo(np.longdouble).eps > 1e-18:
        pytest.skip("long double is not extended precision on this host")
    A = inputs.cfg_small(0)
    res = oracle.run(A, 1e-6, 10, 30, seed=0, mode=1)
    lit = oracle.run(A, 1e-6, 10, 30, seed=0, mode=0)
    assert np.array_equal(res.I, lit.I) and np.array_equal(res.J, lit.J)
    LD = np.longdouble
    G = oracle.gaussian_sketch(0, 30, A.shape[0])
    YL = G.astype(LD) @ A.astype(LD)
    M = A[np.ix_(res.I, res.J)]
    YJ = YL[:, res.J]
    Wt = np.linalg.solve(M.T, YJ.T.astype(np.float64)).astype(LD)
    for _ in range(3):
        Wt = Wt + np.linalg.solve(M.T, (YJ.T - M.T.astype(LD) @ Wt).astype(np.float64)).astype(LD)
    SL = YL - Wt.T @ A[res.I, :].astype(LD)
    rho_ex = float(np.sqrt((SL ** 2).sum() / (YL ** 2).sum()))
    assert abs(res.rho - rho_ex) / rho_ex < 1e-7
    # the literal form (explicit U) is the less accurate of the two here
    assert abs(res.rho - rho_ex) <= abs(lit.rho - rho_ex)


def test_edge_cases():
    A = np.zeros((30, 20))
    res = oracle.run(A, 1e-6, 4, 5, seed=0)
    assert res.rank == 0 and res.rho == 0.0 and res.status == 0
    B = inputs.svd_matrix(30, 20, 0.5 ** np.arange(20), seed=1)
    assert oracle.run(B, 1.0, 4, 5, seed=0).rank == 0          # tol >= rho_0 = 1
    capped = oracle.run(B, 1e-14, 4, 5, seed=0, max_rank=6)
    assert capped.rank == 6 and capped.status == 7               # last block clamped
    wide = oracle.run(B[:7], 1e-12, 4, 5, seed=0)                # m = 7 < 2 b
    assert wide.rank <= 7
    with pytest.raises(ValueError):
        oracle.run(B, 1e-6, 4, 3, seed=0)                        # c < b
