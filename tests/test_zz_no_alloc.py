"""cur_step_lupp_noalloc: the LUPP selection for callers that cannot call
cudaMalloc (framework-owned memory pools, allocation-free loops).  Its scratch
is a fixed device array inside the library, so its result must equal that of
cur_step_lupp, which uses a context workspace, on consecutive calls that reuse
the same array.  Collected last so that a failure here leaves every other test
already run."""
import ctypes

import numpy as np
import pytest

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


def _noalloc(X, steps, mask):
    import paper_2509_21963_gb300 as cur
    nr, ncand = X.shape
    piv = torch.full((steps,), -1, dtype=torch.int64, device=X.device)
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream
    st = cur.lib().cur_step_lupp_noalloc(0, ctypes.c_void_p(stream), ctypes.c_void_p(X.data_ptr()),
                                         X.stride(0), nr, ncand, steps,
                                         ctypes.c_void_p(mask.data_ptr()),
                                         ctypes.c_void_p(piv.data_ptr()), err, len(err))
    return st, piv, err.value.decode()


def test_noalloc_matches_workspace_entry_point_twice(ctx):
    import paper_2509_21963_gb300 as cur
    rng = np.random.default_rng(21)
    # two calls in a row with different shapes: the second reuses the scratch
    for nr, ncand, steps in [(55, 20000, 50), (30, 801, 10)]:
        X = torch.from_numpy(rng.standard_normal((nr, ncand))).cuda()
        mask0 = torch.zeros(ncand, dtype=torch.uint8, device="cuda")
        mask0[torch.from_numpy(rng.choice(ncand, 7, replace=False)).cuda()] = 1
        ref_piv, ref_mask = ctx.lupp(X, steps, mask0.clone())
        m2 = mask0.clone()
        st, piv, msg = _noalloc(X, steps, m2)
        assert st == cur.CUR_OK, msg
        assert torch.equal(piv, ref_piv)          # LUPP pivots: bit-exact
        assert torch.equal(m2, ref_mask)


def test_noalloc_rejects_oversize(ctx):
    import paper_2509_21963_gb300 as cur
    X = torch.zeros((64, 40000), dtype=torch.float64, device="cuda")  # 20 MB > 16 MiB
    mask = torch.zeros(40000, dtype=torch.uint8, device="cuda")
    st, piv, msg = _noalloc(X, 4, mask)
    assert st == cur.CUR_EINVAL and "maximum" in msg


def test_noalloc_largest_problem_that_fits(ctx):
    """The largest candidate count that fits the fixed scratch at nr = 55 (found
    by bisection on the size check, which rejects oversize problems before
    launching; the probes that fit run one step on zeros): it runs and equals
    cur_step_lupp; one more candidate is rejected."""
    import paper_2509_21963_gb300 as cur
    nr, steps = 55, 50
    lo, hi = 20000, 60000                     # fits / does not fit
    mask = torch.zeros(hi + 1, dtype=torch.uint8, device="cuda")
    Xbig = torch.zeros((nr, hi + 1), dtype=torch.float64, device="cuda")
    while hi - lo > 1:
        mid = (lo + hi) // 2
        st, _, msg = _noalloc(Xbig[:, :mid], 1, mask[:mid].zero_())
        if st == cur.CUR_OK:
            lo = mid
        else:
            assert st == cur.CUR_EINVAL and "maximum" in msg, msg
            hi = mid
    X = torch.from_numpy(np.random.default_rng(22).standard_normal((nr, lo))).cuda()
    ref_piv, ref_mask = ctx.lupp(X, steps, torch.zeros(lo, dtype=torch.uint8, device="cuda"))
    m2 = torch.zeros(lo, dtype=torch.uint8, device="cuda")
    st, piv, msg = _noalloc(X, steps, m2)
    assert st == cur.CUR_OK, msg
    assert torch.equal(piv, ref_piv) and torch.equal(m2, ref_mask)
    X1 = torch.zeros((nr, lo + 1), dtype=torch.float64, device="cuda")
    st, _, msg = _noalloc(X1, steps, torch.zeros(lo + 1, dtype=torch.uint8, device="cuda"))
    assert st == cur.CUR_EINVAL and "maximum" in msg
