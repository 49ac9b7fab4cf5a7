"""Serving form (include/cur_server.h): requests against the FP64 oracle, the
same request alone and inside a mix, host-memory requests, admission under a
tight HBM budget, and the server's bookkeeping."""
import time

import numpy as np
import pytest

import oracle
from paper_2509_21963_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_batch_gpu import _check_job  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_21963_gb300 as cur
    c = cur.Context(0)
    yield c
    c.close()


def _requests(k, seed, lo=64, hi=400):
    specs = inputs.batch_specs(k, seed, lo, hi)
    tols = np.random.default_rng(seed).choice([1e-2, 1e-4, 1e-6], size=k)
    mats = [inputs.batch_matrix(s).astype(np.float32) for s in specs]
    return specs, [float(t) for t in tols], mats


@pytest.mark.parametrize("team", [1, 4])
def test_serve_parity(ctx, team):
    """A burst of 16 requests of mixed shapes, spectra and tolerances
    ({1e-2, 1e-4, 1e-6}, b = 10, c = 12), each against the oracle."""
    import paper_2509_21963_gb300 as cur
    specs, tols, mats = _requests(16, seed=21)
    S = cur.Server(ctx, 2 << 30, "float32", team=team, streams=3)
    dev = [torch.from_numpy(A).cuda() for A in mats]
    tickets = [S.submit(A, t, 10, 12, seed=s["seed"]) for A, t, s in zip(dev, tols, specs)]
    S.drain()
    for tk, A, t, s in zip(tickets, mats, tols, specs):
        got = S.result(tk)
        assert got.latency_ms >= got.queue_ms >= 0.0
        A64 = A.astype(np.float64)
        ref = oracle.run(A64, t, 10, 12, seed=s["seed"], mode=1)
        _check_job(A64, got, ref, 10, t)
    st = S.stats()
    assert st["completed"] == st["submitted"] == 16 and st["bytes_in_use"] == 0
    S.close()


def test_serve_alone_equals_in_mix(ctx):
    """A request's result does not depend on the other requests in flight."""
    import paper_2509_21963_gb300 as cur
    specs, tols, mats = _requests(12, seed=5, lo=100, hi=600)
    dev = [torch.from_numpy(A).cuda() for A in mats]
    S = cur.Server(ctx, 4 << 30, "float32", team=2, streams=4)
    probe = 3
    t0 = S.submit(dev[probe], 1e-4, 8, 8, seed=77)
    S.drain()
    alone = S.result(t0)
    tickets = []
    for k in range(len(dev)):  # the probe request submitted in the middle of the mix
        tickets.append(S.submit(dev[k], tols[k], 8, 8, seed=specs[k]["seed"]))
        if k == 6:
            tp = S.submit(dev[probe], 1e-4, 8, 8, seed=77)
    S.drain()
    mixed = S.result(tp)
    assert np.array_equal(alone.I, mixed.I) and np.array_equal(alone.J, mixed.J)
    assert np.array_equal(alone.U, mixed.U) and alone.rho == mixed.rho
    for tk in tickets:
        assert S.result(tk).status in (cur.CUR_OK, cur.CUR_TOL_UNREACHED)
    S.close()


def test_serve_host_requests(ctx):
    """Requests whose A is in host memory give the device requests' results."""
    import paper_2509_21963_gb300 as cur
    specs, tols, mats = _requests(6, seed=8)
    S = cur.Server(ctx, 1 << 30, "float32", team=2, streams=2)
    th = [S.submit(A, t, 8, 8, seed=s["seed"]) for A, t, s in zip(mats, tols, specs)]
    dev = [torch.from_numpy(A).cuda() for A in mats]
    td = [S.submit(A, t, 8, 8, seed=s["seed"]) for A, t, s in zip(dev, tols, specs)]
    S.drain()
    for a, b in zip(th, td):
        ra, rb = S.result(a), S.result(b)
        assert np.array_equal(ra.I, rb.I) and np.array_equal(ra.U, rb.U) and ra.rho == rb.rho
    S.close()


def test_serve_admission_budget(ctx):
    """A budget that holds about two requests at a time: everything still
    completes, the arena never exceeds the budget, and requests queue."""
    import paper_2509_21963_gb300 as cur
    A = inputs.batch_matrix(dict(m=600, n=500, kind="poly1.5", r=0, seed=3)).astype(np.float32)
    Ad = torch.from_numpy(A).cuda()
    budget = 30 << 20  # one request needs ~12.6 MB
    S = cur.Server(ctx, budget, "float32", team=2, streams=2)
    tickets = [S.submit(Ad, 1e-4, 8, 8, seed=k) for k in range(6)]
    results = []
    for tk in tickets:  # release each result as it arrives so later ones can be admitted
        S.wait(tk)
        results.append(S.result(tk))
    st = S.stats()
    assert st["bytes_peak"] <= budget and st["completed"] == 6 and st["bytes_in_use"] == 0
    assert max(r.queue_ms for r in results) > 0.0
    ref = oracle.run(A.astype(np.float64), 1e-4, 8, 8, seed=0, mode=1)
    _check_job(A.astype(np.float64), results[0], ref, 8, 1e-4)
    S.close()


def test_serve_errors(ctx):
    import paper_2509_21963_gb300 as cur
    S = cur.Server(ctx, 16 << 20, "float32", team=1, streams=1)
    big = torch.zeros(2000, 2000, dtype=torch.float32, device="cuda")
    with pytest.raises(cur.CurError) as e:
        S.submit(big, 1e-4, 8, 8)
    assert e.value.status == cur.CUR_EBUDGET
    small = torch.zeros(40, 30, dtype=torch.float32, device="cuda")
    with pytest.raises(cur.CurError) as e:
        S.submit(small, 1e-4, 0, 8)
    assert e.value.status == cur.CUR_EINVAL
    with pytest.raises(TypeError):
        S.submit(small.double(), 1e-4, 4, 4)
    tk = S.submit(small, 1e-4, 4, 4)  # an all-zero matrix: rank 0, rho 0
    S.wait(tk, 30.0)
    r = S.result(tk)
    assert r.rank == 0 and r.rho == 0.0 and r.status == cur.CUR_OK
    with pytest.raises(cur.CurError):
        S.result(tk)  # released with the result
    S.close()
    with pytest.raises(cur.CurError):
        cur.Server(ctx, 1 << 30, "float32", team=9)
    with pytest.raises(cur.CurError):
        cur.Server(ctx, 1 << 30, "float32", team=2, big_lanes=5)


def test_serve_large_requests_alone(ctx):
    """Requests at or above the size threshold run alone through the
    single-matrix path: the same result as cur_run on the caller's context,
    with small requests served before and after them."""
    import paper_2509_21963_gb300 as cur
    specs, tols, mats = _requests(8, seed=31, lo=64, hi=300)
    big = inputs.batch_matrix(dict(m=900, n=700, kind="exp20", r=0, seed=4)).astype(np.float32)
    S = cur.Server(ctx, 2 << 30, "float32", team=2, streams=2, big_elements=500_000, big_lanes=2)
    dev = [torch.from_numpy(A).cuda() for A in mats]
    bd = torch.from_numpy(big).cuda()
    tickets = [S.submit(A, t, 8, 8, seed=s["seed"]) for A, t, s in zip(dev[:4], tols, specs)]
    tb = S.submit(bd, 1e-6, 50, 55, seed=9)
    th = S.submit(big, 1e-6, 50, 55, seed=9)  # the same large request from host memory
    tb2 = S.submit(bd, 1e-6, 50, 55, seed=9)  # two lanes: these run at the same time
    # a large request of another shape and block size beside them: its kernels
    # launch with other shared-memory sizes while the first ones are in flight
    other = inputs.batch_matrix(dict(m=640, n=1100, kind="exp20", r=0, seed=6)).astype(np.float32)
    od = torch.from_numpy(other).cuda()
    to = [S.submit(od, 1e-6, 20, 24, seed=k) for k in range(3)]
    tickets += [S.submit(A, t, 8, 8, seed=s["seed"]) for A, t, s in zip(dev[4:], tols[4:], specs[4:])]
    S.drain()
    for k, t in enumerate(to):
        got, want = S.result(t), ctx.run(od, 1e-6, 20, 24, k)
        assert got.status == cur.CUR_OK, got.error
        assert np.array_equal(got.I, want.I) and np.array_equal(got.U, want.U)
    ref_run = ctx.run(bd, 1e-6, 50, 55, 9)
    for t in (tb, th, tb2):
        got = S.result(t)
        assert np.array_equal(got.I, ref_run.I) and np.array_equal(got.J, ref_run.J)
        assert np.array_equal(got.U, ref_run.U) and got.rho == ref_run.rho
        assert np.array_equal(got.rho_history, ref_run.rho_history)
    big64 = big.astype(np.float64)
    ref = oracle.run(big64, 1e-6, 50, 55, seed=9, mode=1)
    _check_job(big64, ref_run, ref, 50, 1e-6)
    for tk, A, t, s in zip(tickets, mats, tols, specs):
        got = S.result(tk)
        A64 = A.astype(np.float64)
        _check_job(A64, got, oracle.run(A64, t, 8, 8, seed=s["seed"], mode=1), 8, t)
    assert S.stats()["bytes_in_use"] == 0
    S.close()
