"""The measurement probes of include/cur_steps.h: the FP64 FMA rate and the
per-operation latencies return plausible values (positive, a divide slower
than one FMA, one FMA no faster with a single active lane)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_probes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_21963_gb300 as cur
    ctx = cur.Context(0)
    try:
        assert 0.1 < ctx.fp64_tflops() < 100.0
        lat = ctx.latency_cycles()
        assert all(v > 0 for v in lat.values()), lat
        assert lat["ddiv"] > lat["dfma"] and lat["dsqrt_add"] > lat["dfma"]
        assert lat["dfma_one_lane"] >= 0.5 * lat["dfma"]
        assert lat["l2_load"] > lat["ffma"]
    finally:
        ctx.close()
