"""Batched form (include/cur_batch.h): every job of one persistent launch
against the FP64 oracle run on the same matrix with the same (tol, b, c, seed).

The per-job gates are those of the single-matrix path (test_parity_gpu):
indices bit-exact over the oracle's decided selections, rho within the derived
rounding bound, U within the pivoted-QR backward-error bound.  Jobs whose
later selections are at rounding level in the oracle (exact-rank jobs once the
rank is exhausted) are compared over the decided prefix and must still meet
the tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_2509_21963_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_parity_gpu import _check_parity, _decided_prefix  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_21963_gb300 as cur
    c = cur.Context(0)
    yield c
    c.close()


def _jobs(njobs, seed, lo, hi, dtype):
    specs = inputs.batch_specs(njobs, seed, lo, hi)
    mats64 = [inputs.batch_matrix(s) for s in specs]
    if dtype == torch.float32:
        mats64 = [A.astype(np.float32).astype(np.float64) for A in mats64]
    dev = [torch.from_numpy(A).to(dtype).cuda() for A in mats64]
    return specs, mats64, dev


def _check_job(A, got, ref, b, tol):
    n_dec = _decided_prefix(ref, b, ref.maxabsY)
    _check_parity(A, got, ref, b, require_full=False)
    if n_dec < ref.rank:
        # selections at rounding level: the result must still be valid, and its
        # CUR as accurate as the oracle's (with an ill-conditioned core the FP64
        # U = A(I,J)^+ limits both: e.g. 1.3e-6 at tol 1e-10 on s_i = 0.5^i)
        assert got.status == 0 and got.rho <= tol
        e_g = oracle.true_error(A, got.I, got.J, got.U)
        e_o = oracle.true_error(A, ref.I, ref.J, ref.U)
        assert e_g <= max(10 * tol, 4 * e_o), (e_g, e_o)
    return n_dec == ref.rank


@pytest.mark.parametrize("dtype,team", [(torch.float64, 1), (torch.float64, 4),
                                        (torch.float32, 2), (torch.float32, 8)])
def test_batch_parity(ctx, dtype, team):
    """24 jobs, m, n log-uniform in [16, 200], mixed spectra, tol 1e-4, b = c = 8
    (the batched workload's parameters at oracle-friendly sizes)."""
    import paper_2509_21963_gb300 as cur
    specs, mats, dev = _jobs(24, seed=7, lo=16, hi=200, dtype=dtype)
    B = cur.Batch(ctx, dev, 1e-4, 8, 8, seed=[s["seed"] for s in specs])
    B.set_team(team)
    B.run()
    full = 0
    for j, (s, A) in enumerate(zip(specs, mats)):
        ref = oracle.run(A, 1e-4, 8, 8, seed=s["seed"], mode=1)
        got = B.result(j)
        full += _check_job(A, got, ref, 8, 1e-4)
    assert full == len(specs)   # every job's oracle selection is decided: compared in full
    B.close()


def test_batch_tile_4_equals_tile_8(ctx):
    """The product tile changes registers and reuse, not the arithmetic: the
    batch gives the same I, J, U and rho bit for bit with tiles of 4 and 8."""
    import paper_2509_21963_gb300 as cur
    specs, mats, dev = _jobs(12, seed=19, lo=30, hi=220, dtype=torch.float64)
    B = cur.Batch(ctx, dev, 1e-4, 8, 8, seed=[s["seed"] for s in specs])
    B.set_team(2)
    B.run()
    r8 = [B.result(j) for j in range(len(specs))]
    B.set_tile(4)
    assert B.schedule()["tile_n"] == 4
    B.run()
    for j in range(len(specs)):
        a, b = r8[j], B.result(j)
        assert np.array_equal(a.I, b.I) and np.array_equal(a.J, b.J)
        assert np.array_equal(a.U, b.U) and a.rho == b.rho
    with pytest.raises(cur.CurError):
        B.set_tile(6)
    B.close()


@pytest.mark.parametrize("team,team_big,nbig,cut", [(1, 8, 1, 3), (2, 16, 2, 6), (4, 8, 2, 23)])
def test_batch_team_classes(ctx, team, team_big, nbig, cut):
    """Two team classes in one launch (big teams take the `cut` largest jobs
    first, then help with the rest): every job against the oracle over its
    whole selection, as in test_batch_parity."""
    import paper_2509_21963_gb300 as cur
    specs, mats, dev = _jobs(24, seed=7, lo=16, hi=200, dtype=torch.float64)
    B = cur.Batch(ctx, dev, 1e-4, 8, 8, seed=[s["seed"] for s in specs])
    B.set_classes(team, team_big, nbig, cut)
    sch = B.schedule()
    assert (sch["team"], sch["team_big"], sch["nbig"], sch["big_cut"]) == (team, team_big, nbig, cut)
    assert sch["teams"] == nbig + (sch["grid"] - nbig * team_big) // team
    B.run()
    full = 0
    for j, (s, A) in enumerate(zip(specs, mats)):
        ref = oracle.run(A, 1e-4, 8, 8, seed=s["seed"], mode=1)
        full += _check_job(A, B.result(j), ref, 8, 1e-4)
    assert full == len(specs)
    with pytest.raises(cur.CurError):
        B.set_classes(team, 32, 64, cut)   # no room left for a small team
    B.close()


def test_batch_other_block_sizes(ctx):
    """Jobs with different b and c in one batch (b up to 64, c up to 128)."""
    import paper_2509_21963_gb300 as cur
    rng = np.random.default_rng(3)
    cases = [(5, 7), (16, 20), (1, 1), (3, 30), (64, 128), (32, 35)]
    mats, dev = [], []
    for k, (b, c) in enumerate(cases):
        m, n = int(rng.integers(70, 220)), int(rng.integers(70, 220))
        A = inputs.svd_matrix(m, n, 10.0 ** (-np.arange(1, min(m, n) + 1) / 12.0), seed=40 + k)
        mats.append(A)
        dev.append(torch.from_numpy(A).cuda())
    B = cur.Batch(ctx, dev, 1e-6, [b for b, _ in cases], [c for _, c in cases],
                  seed=list(range(len(cases))))
    B.run()
    for j, (b, c) in enumerate(cases):
        ref = oracle.run(mats[j], 1e-6, b, c, seed=j, mode=1)
        _check_job(mats[j], B.result(j), ref, b, 1e-6)
    B.close()


def test_batch_edge_cases(ctx):
    """Zero matrix, tol >= 1, a matrix thinner than b, a rank cap, a NaN entry,
    and ordinary jobs next to them."""
    import paper_2509_21963_gb300 as cur
    A1 = inputs.svd_matrix(60, 50, 0.5 ** np.arange(50), seed=1)
    A2 = inputs.svd_matrix(3, 90, np.array([1.0, 0.3, 0.01]), seed=2)
    bad = A1.copy()
    bad[3, 7] = np.nan
    mats = [np.zeros((40, 30)), A1, A1, A2, A1, bad, A1]
    tols = [1e-6, 1.0, 1e-14, 1e-12, 1e-6, 1e-6, 1e-10]
    mr = [0, 0, 6, 0, 0, 0, 0]
    dev = [torch.from_numpy(A).cuda() for A in mats]
    B = cur.Batch(ctx, dev, tols, 4, 5, seed=0, max_rank=mr)
    B.run()
    r = B.result(0)
    assert r.rank == 0 and r.rho == 0.0 and r.status == 0
    r = B.result(1)
    assert r.rank == 0 and r.rho == 1.0 and r.status == 0
    r = B.result(2)
    ref = oracle.run(A1, 1e-14, 4, 5, seed=0, max_rank=6, mode=1)
    assert r.rank == 6 and r.status == cur.CUR_TOL_UNREACHED
    assert np.array_equal(r.I, ref.I) and np.array_equal(r.J, ref.J)
    r = B.result(3)
    ref = oracle.run(A2, 1e-12, 4, 5, seed=0, mode=1)
    assert r.rank == ref.rank == 3
    assert np.array_equal(r.I, ref.I) and np.array_equal(r.J, ref.J)
    r = B.result(5)
    assert r.status == cur.CUR_ENONFINITE and r.rank == 0
    for j in (4, 6):
        ref = oracle.run(A1, tols[j], 4, 5, seed=0, mode=1)
        _check_job(A1, B.result(j), ref, 4, tols[j])
    B.close()


def test_batch_repeat_is_deterministic(ctx):
    """Two launches of the same batch (graph replay when available) give
    bitwise-identical results."""
    import paper_2509_21963_gb300 as cur
    specs, mats, dev = _jobs(10, seed=11, lo=20, hi=150, dtype=torch.float32)
    B = cur.Batch(ctx, dev, 1e-4, 8, 8, seed=[s["seed"] for s in specs])
    B.set_team(2)
    B.run()
    first = [B.result(j) for j in range(len(specs))]
    B.run()
    for j in range(len(specs)):
        r = B.result(j)
        assert np.array_equal(r.I, first[j].I) and np.array_equal(r.J, first[j].J)
        assert np.array_equal(r.U, first[j].U) and r.rho == first[j].rho
    B.close()


def test_batch_tune(ctx):
    import paper_2509_21963_gb300 as cur
    specs, mats, dev = _jobs(12, seed=5, lo=32, hi=256, dtype=torch.float32)
    B = cur.Batch(ctx, dev, 1e-4, 8, 8, seed=[s["seed"] for s in specs])
    team, ms = B.tune([1, 2, 4])
    assert team in (1, 2, 4) and ms > 0
    assert B.schedule()["team"] == team
    for j in (0, 5, 11):
        ref = oracle.run(mats[j], 1e-4, 8, 8, seed=specs[j]["seed"], mode=1)
        _check_job(mats[j], B.result(j), ref, 8, 1e-4)
    B.close()


def test_batch_argument_errors(ctx):
    import paper_2509_21963_gb300 as cur
    A = torch.zeros(32, 32, dtype=torch.float64, device="cuda")
    for kw in [dict(block_size=0), dict(block_size=65), dict(block_size=8, sketch_size=7),
               dict(block_size=8, sketch_size=129), dict(block_size=4, tol=0.0),
               dict(block_size=4, tol=float("nan"))]:
        tol = kw.pop("tol", 1e-3)
        with pytest.raises(cur.CurError) as e:
            cur.Batch(ctx, [A, A], tol, **kw)
        assert e.value.status == cur.CUR_EINVAL and "job 0" in str(e.value)
    with pytest.raises(TypeError):
        cur.Batch(ctx, [A, A.float()], 1e-3, 4)


@pytest.mark.parametrize("team", [1, 4])
def test_batch_large_cores(ctx, team):
    """Cores larger than a CTA's 256 threads (p up to 650), where each thread of
    the core solve owns several rows: against the oracle, and bitwise equal on
    a second launch (a cross-thread race would show as run-to-run noise)."""
    import paper_2509_21963_gb300 as cur
    cases = [(520, 400, "poly1.5", 1e-4, 8, 8), (300, 610, "exp20", 1e-6, 8, 8),
             (700, 650, "poly1.5", 1e-4, 16, 20), (306, 270, "exp20", 1e-6, 10, 12)]
    mats, dev = [], []
    for k, (m, n, kind, *_rest) in enumerate(cases):
        A = inputs.batch_matrix(dict(m=m, n=n, kind=kind, r=0, seed=90 + k))
        mats.append(A)
        dev.append(torch.from_numpy(A).cuda())
    B = cur.Batch(ctx, dev, [c[3] for c in cases], [c[4] for c in cases], [c[5] for c in cases],
                  seed=list(range(len(cases))))
    B.set_team(team)
    B.run()
    first = [B.result(j) for j in range(len(cases))]
    B.run()
    for j, (m, n, kind, tol, b, c) in enumerate(cases):
        got = B.result(j)
        assert np.array_equal(got.U, first[j].U) and got.rho == first[j].rho
        ref = oracle.run(mats[j], tol, b, c, seed=j, mode=1)
        assert ref.rank > 256
        _check_job(mats[j], got, ref, b, tol)
    B.close()
