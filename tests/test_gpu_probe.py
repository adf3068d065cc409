"""libdotprobe on the GPU: every probe runs and reports its units, and the
tensor-pipe shapes of the fixed-operand multiply run at a plausible rate:
above a third of the chip's nominal dense fp16 rate and not far above it."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_21566_gb300 import probe
    probe.lib()
    return probe


def test_every_probe_runs(P):
    for kind in (P.MUL_PAIR, P.COLSUM_R8, P.MADWIDE_R8, P.MUL_LO, P.EMPTY):
        ms, units = P.run(kind, 4, 16, reps=2)
        assert ms > 0 and units > 0


def test_tensor_pipe_shapes(P):
    sms, per = P.occupancy(P.MMA_N128_TMEM)
    assert per == 1
    nominal = 2.25e15 * sms / 152   # nominal dense fp16 of a 152-SM GB300, scaled to this SM count
    for kind in (P.MMA_N128_TMEM, P.MMA_N128_SMEM, P.MMA_N256_TMEM):
        iters = 20000
        ms, units = P.run(kind, sms, iters, reps=3)
        n = 256 if kind == P.MMA_N256_TMEM else 128
        assert units == 2.0 * 128 * n * 16 * 4 * iters * sms
        rate = units / (ms * 1e-3)
        assert nominal / 3 < rate < nominal * 1.15, (kind, rate)
