"""Pins of the oracle's precision-form functions (CPU only).

The tensor-core forms of the sketch are defined by functions of this project,
not of the paper: the 8-bit rounding of the Gaussian sketch, the S-digit fixed
point of the precision forms, and the exact 52-bit fixed-point sketch of the
FP64 tensor-core form.  Each is pinned here to the mathematics it states (a
closed-form error bound, exactness on values already on the grid, the column
scale from an independent frexp, an exact rational evaluation with Python
integers, a library product on integer data), chosen so that a wrong rounding
(ties, truncation vs rounding), an off-by-one column exponent, a wrong digit
sign or a dropped digit fails at least one test.  The loop entry points that
take a given sketch are pinned to the plain run bit for bit, and the true
error to a direct numpy evaluation (Sec. 3.3 defines rho against it).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2509_21963_gb300 import inputs


def _frexp_exp(col):
    mx = float(np.max(np.abs(col))) if col.size else 0.0
    return math.frexp(mx)[1] if mx > 0 else 0


def _adversarial_columns(rng, m):
    cols = [
        rng.standard_normal(m),                                   # generic
        np.zeros(m),                                              # zero column
        np.r_[2.0 ** 5, rng.uniform(-31, 31, m - 1)],             # max an exact power of two
        np.r_[-(2.0 ** -7), rng.uniform(-2 ** -8, 2 ** -8, m - 1)],  # negative power-of-two max
        rng.standard_normal(m) * 10.0 ** rng.uniform(-9, 0, m),   # 1e9 dynamic range
        np.full(m, 3.0),                                          # constant
    ]
    # half-digit ties at the lowest digit of S = 2 (scale 2^E, E = 1): the grid
    # is 2^(1 - 16); entries k + 1/2 grid units
    g = 2.0 ** (1 - 16)
    ties = (np.arange(m) % 7 + 0.5) * g
    ties[0] = 1.5                                                 # max 1.5 -> E = 1
    cols.append(ties)
    return np.stack(cols, axis=1)


# --------------------------------------------------------------------------
# fix_S of the precision forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("S", [1, 2, 3, 4])
def test_fixed_point_error_bound_and_grid(S):
    rng = np.random.default_rng(S)
    A = _adversarial_columns(rng, 64)
    F = oracle.fixed_point(A, S)
    for j in range(A.shape[1]):
        E = _frexp_exp(A[:, j])
        grid = 2.0 ** (E - 8 * S)
        # |fix_S(x) - x| <= 2^(E - 8S - 1): round to nearest on the grid
        assert np.all(np.abs(F[:, j] - A[:, j]) <= grid / 2)
        # the result is on the grid 2^(E - 8S) and within the S-digit range
        v = F[:, j] / grid
        assert np.all(v == np.round(v)) and np.all(np.abs(v) <= 2.0 ** (8 * S))
        # values already on the grid are unchanged
        on = np.round(A[:, j] / grid) * grid
        if np.max(np.abs(on)) > 0 and _frexp_exp(on) == E:
            np.testing.assert_array_equal(oracle.fixed_point(on[:, None], S)[:, 0], on)


@pytest.mark.parametrize("S", [1, 2, 3, 4])
def test_fixed_point_is_one_rounding_half_even(S):
    """The digit recursion equals a single rounding of x 2^(8S-E) to the
    nearest integer, ties to even, with E from an independent frexp of the
    column max (exact rational arithmetic in Python)."""
    rng = np.random.default_rng(10 + S)
    A = _adversarial_columns(rng, 48)
    F = oracle.fixed_point(A, S)
    for j in range(A.shape[1]):
        E = _frexp_exp(A[:, j])
        for k in range(A.shape[0]):
            v = round(Fraction(float(A[k, j])) * Fraction(2) ** (8 * S - E))  # half to even
            assert F[k, j] == float(Fraction(v) * Fraction(2) ** (E - 8 * S)), (S, j, k)


def test_fixed_point_ties_go_to_even():
    """A column max of 1.5 gives E = 1, grid 2^-15 for S = 2; entries at k + 1/2
    grid units round to the even neighbour (2.5 -> 2, 3.5 -> 4, -0.5 -> 0)."""
    g = 2.0 ** -15
    col = np.array([1.5, 2.5 * g, 3.5 * g, -0.5 * g, 0.5 * g, -1.5 * g])
    F = oracle.fixed_point(col[:, None], 2)[:, 0] / g
    np.testing.assert_array_equal(F[1:], [2.0, 4.0, 0.0, 0.0, -2.0])


@pytest.mark.parametrize("S", [1, 2, 3, 4])
def test_fixed_point_digits(S):
    """Every digit is an integer with |d| <= 256 (exact in BF16; the leading
    one up to 256, the others |d| <= 128 after a round to nearest), and the
    digits reassemble the oracle's fix_S value."""
    rng = np.random.default_rng(20 + S)
    A = _adversarial_columns(rng, 40)
    F = oracle.fixed_point(A, S)
    for j in range(A.shape[1]):
        E = _frexp_exp(A[:, j])
        for k in range(A.shape[0]):
            d = oracle.fixed_point_digits(A[k, j], E, S)
            assert np.all(d == np.round(d))
            assert abs(d[S - 1]) <= 256 and np.all(np.abs(d[:S - 1]) <= 128)
            v = sum(int(d[s]) * 256 ** s for s in range(S))
            assert F[k, j] == math.ldexp(v, E - 8 * S)


def test_fixed_point_exponent_matches_frexp():
    """E_j is frexp of the column max: the column max itself keeps its leading
    digit below 256 (x 2^(8-E) in [128, 256)), and doubling the max moves the
    grid by one binade (a column of 2^k and 2^k - 2^(k-30))."""
    for k in (-20, -1, 0, 3, 40):
        col = np.array([2.0 ** k, 2.0 ** k - 2.0 ** (k - 30)])
        E = math.frexp(2.0 ** k)[1]
        assert E == k + 1
        d = oracle.fixed_point_digits(col[0], E, 1)
        assert d[0] == 128.0
        # one digit: 2^k - 2^(k-30) rounds to the same digit 128
        assert oracle.fixed_point(col[:, None], 1)[1, 0] == 2.0 ** k


# --------------------------------------------------------------------------
# 8-bit Gaussian sketch
# --------------------------------------------------------------------------
def test_gaussian_q8_is_rounded_gaussian():
    c, m, seed = 7, 30000, 5
    Q = oracle.gaussian_sketch_q8(seed, c, m)
    Z = oracle.gaussian_sketch(seed, c, m)
    assert np.all(Q == np.round(Q)) and np.all(np.abs(Q) <= 127)
    inside = np.abs(16 * Z) <= 127.5
    assert np.all(np.abs(Q[inside] - 16 * Z[inside]) <= 0.5)
    assert np.all(Q[~inside] == 127 * np.sign(Z[~inside]))
    # 16 Z exceeds 127.5 only beyond 7.97 sigma: none in 2.1e5 draws
    assert inside.all()
    # the sketch keeps the Gaussian's moments (variance 256 + 1/12 of rounding)
    assert abs(Q.mean()) < 5 * 16 / math.sqrt(Q.size)
    assert abs(Q.var() / (256 + 1 / 12) - 1) < 5 * math.sqrt(2 / Q.size)


def test_quantize_q8_clamp_and_ties():
    """An explicit sketch beyond 127/16 clamps to +-127; 16 g at k + 1/2 rounds
    to the even neighbour."""
    G = np.array([7.96875, 7.99, 100.0, -8.0, -1e300, 0.03125, 0.09375, -0.03125, 0.0])
    np.testing.assert_array_equal(oracle.quantize_q8(G),
                                  [127, 127, 127, -127, -127, 0, 2, 0, 0])


# --------------------------------------------------------------------------
# exact 52-bit fixed-point sketch (FP64 tensor-core form)
# --------------------------------------------------------------------------
def _fx_matrix(rng, m):
    cols = [
        rng.standard_normal(m),
        np.zeros(m),
        np.r_[2.0 ** 9, rng.uniform(-511, 511, m - 1)],           # power-of-two max
        rng.standard_normal(m) * 10.0 ** rng.uniform(-12, 3, m),  # wide range
        np.r_[1e-310, -3e-312, rng.uniform(-1e-309, 1e-309, m - 2)],  # subnormals only
        np.r_[1.0, 5e-324, -1e-310, np.zeros(m - 3)],             # subnormals in a normal column
        np.r_[-0.0, rng.integers(-1000, 1000, m - 1).astype(np.float64)],
        np.r_[2.0 ** 1000, rng.standard_normal(m - 1) * 2.0 ** 990],  # huge
    ]
    return np.stack(cols, axis=1)


def _fx_exact(Gq, A, Q):
    """Python integers: X = trunc(x 2^(Q-E)), V = sum Gq X, RN(V) 2^(E-Q)."""
    c, m = Gq.shape
    n = A.shape[1]
    Y = np.empty((c, n))
    for j in range(n):
        E = _frexp_exp(A[:, j])
        X = [math.trunc(Fraction(float(a)) * Fraction(2) ** (Q - E)) for a in A[:, j]]
        for i in range(c):
            V = sum(int(Gq[i, k]) * X[k] for k in range(m))
            Y[i, j] = math.ldexp(float(V), E - Q)   # int -> float rounds to nearest even
    return Y


def test_sketch_fx_exact_rational():
    rng = np.random.default_rng(31)
    m, c = 97, 5
    A = _fx_matrix(rng, m)
    Gq = oracle.gaussian_sketch_q8(7, c, m)
    Y = oracle.sketch_fx(Gq, A)
    np.testing.assert_array_equal(Y, _fx_exact(Gq, A, 52))


def test_sketch_fx_error_bound():
    """|Y - Gq A| <= sum_k |Gq| 2^(E-Q) (truncation onto the grid) + half an ulp
    of Y (one rounding), with Gq A evaluated exactly."""
    rng = np.random.default_rng(32)
    m, c = 200, 6
    A = _fx_matrix(rng, m)
    Gq = oracle.gaussian_sketch_q8(8, c, m)
    Y = oracle.sketch_fx(Gq, A)
    for j in range(A.shape[1]):
        E = _frexp_exp(A[:, j])
        for i in range(c):
            exact = sum(Fraction(int(Gq[i, k])) * Fraction(float(A[k, j])) for k in range(m))
            err = abs(Fraction(float(Y[i, j])) - exact)
            bound = Fraction(int(np.abs(Gq[i]).sum())) * Fraction(2) ** (E - 52) + \
                Fraction(float(np.spacing(abs(Y[i, j])))) / 2
            assert err <= bound, (i, j)


def test_sketch_fx_exact_on_grid_data_and_truncates():
    """Integer data (on the grid) gives numpy's exact integer product; an entry
    1.75 grid units above zero truncates to one unit (toward zero: a rounding
    or a floor would give 2 or -2 for its negative)."""
    rng = np.random.default_rng(33)
    A = rng.integers(-2 ** 20, 2 ** 20, size=(300, 9)).astype(np.float64)
    Gq = oracle.gaussian_sketch_q8(9, 4, 300)
    ref = Gq.astype(np.int64) @ A.astype(np.int64)
    np.testing.assert_array_equal(oracle.sketch_fx(Gq, A), ref.astype(np.float64))
    E = 3                                   # column max 7 < 2^3
    g = 2.0 ** (E - 52)
    A = np.array([[7.0, 7.0], [1.75 * g, -1.75 * g]])
    Y = oracle.sketch_fx(np.array([[0.0, 1.0]]), A)
    np.testing.assert_array_equal(Y, [[g, -g]])


def test_sketch_fx_nonfinite_column():
    A = np.ones((4, 3))
    A[2, 1] = np.inf
    Y = oracle.sketch_fx(np.ones((2, 4)), A)
    assert np.all(np.isnan(Y[:, 1])) and np.all(Y[:, [0, 2]] == 4.0)


# --------------------------------------------------------------------------
# loops started from a given sketch; the true error
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
def test_run_sketched_of_A_equals_run(mode):
    A = inputs.cfg_small(4)[:300, :200].copy()
    a = oracle.run(A, 1e-6, 8, 12, seed=2, mode=mode)
    b = oracle.run(A, 1e-6, 8, 12, seed=2, mode=mode, A_sketch=A)
    assert np.array_equal(a.I, b.I) and np.array_equal(a.J, b.J)
    assert a.rho == b.rho and np.array_equal(a.rho_hist, b.rho_hist)
    assert np.array_equal(a.U, b.U)


def test_run_y_equals_run_with_its_sketch():
    A = inputs.cfg_small(5)[:300, :200].copy()
    G = oracle.gaussian_sketch(6, 12, 300)
    a = oracle.run(A, 1e-6, 8, 12, G=G, mode=1)
    b = oracle.run_y(A, 1e-6, 8, 12, oracle.sketch(G, A), mode=1)
    assert np.array_equal(a.I, b.I) and np.array_equal(a.J, b.J)
    assert a.rho == b.rho and np.array_equal(a.U, b.U)


def test_run_fx_recovers_exact_rank():
    """The FP64 tensor-core form (8-bit sketch, 52-bit fixed point) keeps
    Sec. 5.1's exact-rank recovery: true error and rho at rounding level once
    r indices are chosen."""
    A = inputs.exact_rank(400, 300, 25, seed=6)
    r = oracle.run_fx(A, 1e-11, 10, 12, seed=4)
    assert r.status == 0 and r.rank == 30
    assert oracle.true_error(A, r.I, r.J, r.U) < 1e-12 and r.rho < 1e-11


def test_true_error_matches_numpy():
    rng = np.random.default_rng(40)
    A = rng.standard_normal((60, 45))
    I = rng.choice(60, 7, replace=False)
    J = rng.choice(45, 7, replace=False)
    U = np.linalg.inv(A[np.ix_(I, J)])
    ref = np.linalg.norm(A - A[:, J] @ U @ A[I, :]) / np.linalg.norm(A)
    assert abs(oracle.true_error(A, I, J, U) - ref) <= 1e-13 * max(ref, 1.0)
    # U^T or swapped roles change the value
    assert abs(oracle.true_error(A, I, J, U.T) - ref) > 1e-3


def test_threads_do_not_change_results():
    """The oracle's parallel loops are independent outer loops (no split
    reduction): one thread and many give bit-identical runs."""
    A = inputs.cfg_small(6)
    t = oracle.threads()
    try:
        oracle.set_threads(1)
        a = oracle.run_fx(A, 1e-6, 10, 30, seed=1)
        b = oracle.run(A, 1e-6, 10, 30, seed=1, mode=0)
        oracle.set_threads(max(t, 4))
        c = oracle.run_fx(A, 1e-6, 10, 30, seed=1)
        d = oracle.run(A, 1e-6, 10, 30, seed=1, mode=0)
    finally:
        oracle.set_threads(t)
    assert np.array_equal(a.I, c.I) and np.array_equal(a.J, c.J)
    assert np.array_equal(a.rho_hist, c.rho_hist) and np.array_equal(a.U, c.U)
    assert np.array_equal(b.I, d.I) and np.array_equal(b.rho_hist, d.rho_hist)
    assert np.array_equal(b.U, d.U)
