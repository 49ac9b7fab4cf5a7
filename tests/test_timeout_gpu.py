"""The failure path of the bounded device waits, driven on purpose without a
fault or a hang: a software grid barrier that expects one CTA more than the
launch has, and an mbarrier phase that gets one of its two arrivals.  Each
wait gives up after a few milliseconds, records the timeout in the status
word and returns; the call reports CUR_ETIMEOUT and the same context then runs
the method normally."""
import time

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


@pytest.mark.parametrize("which,nblocks", [(0, 1), (0, 8), (1, 1)])
def test_bounded_wait_times_out_and_context_survives(ctx, which, nblocks):
    import paper_2509_21963_gb300 as cur
    t0 = time.perf_counter()
    st = ctx.wait_timeout_status(which, nblocks, budget_ms=3.0)
    dt = time.perf_counter() - t0
    assert st == cur.CUR_ETIMEOUT, ctx.last_error()
    assert "budget" in ctx.last_error()
    assert dt < 5.0                       # gave up after its budget, not at a watchdog
    # the same context runs the method afterwards, with the oracle's result
    A = inputs.cfg_small(0)
    ref = oracle.run(A, 1e-6, 10, 30, seed=0, mode=1)
    got = ctx.run(torch.from_numpy(A).cuda(), 1e-6, 10, 30, 0)
    assert got.status == 0 and np.array_equal(got.I, ref.I) and np.array_equal(got.J, ref.J)


def test_timeout_hook_rejects_bad_arguments(ctx):
    import paper_2509_21963_gb300 as cur
    assert ctx.wait_timeout_status(2, 1, 1.0) == cur.CUR_EINVAL
    assert ctx.wait_timeout_status(0, 0, 1.0) == cur.CUR_EINVAL
    assert ctx.wait_timeout_status(0, 1, 0.0) == cur.CUR_EINVAL
    assert ctx.wait_timeout_status(0, 1, 9000.0) == cur.CUR_EINVAL
