"""Autotuner: the persistent cache (CPU) and tuned shapes on the GPU."""
import numpy as np
import pytest

import oracle
from paper_2604_21566_gb300 import tuning
from paper_2604_21566_gb300 import workloads as W


class FakeCtx:
    def __init__(self):
        self.table = {}

    def tune_set(self, op, m, value):
        self.table[(op, int(m).bit_length())] = value

    def autotune(self, op, m, batch):
        return 8, 1.25


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "t.json")
    ctx = FakeCtx()
    knob, ms = tuning.tune(ctx, "GB300", 152, 2, 300, 1000, path=path)
    assert (knob, ms) == (8, 1.25)
    entries = tuning.load(path)
    assert tuning.key("GB300", 152, 2, 300) in entries
    other = FakeCtx()
    assert tuning.apply(other, "GB300", 152, entries) == 1
    assert other.table == {(2, 9): 8}
    # another GPU model or SM count does not pick it up
    assert tuning.apply(FakeCtx(), "GB200", 152, entries) == 0
    assert tuning.apply(FakeCtx(), "GB300", 148, entries) == 0


@pytest.mark.gpu
def test_autotune_and_tuned_parity():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from gpu_util import assert_same, dev, host
    from paper_2604_21566_gb300 import dot
    ctx = dot.Context()
    try:
        knob, ms = ctx.autotune(dot.OP_MUL, 200, 4096)
        assert knob in (8, 12, 16) and ms > 0
        assert ctx.tune_get(dot.OP_MUL, 200) == knob
        knob, ms = ctx.autotune(dot.OP_ADD, 1 << 15, 16)
        assert knob in (1, 2, 4)
        assert ctx.autotune(dot.OP_ADD, 128, 16)[0] == 0      # nothing to tune
        with pytest.raises(dot.DotError):
            ctx.tune_set(dot.OP_MUL, 300, 4)                  # R = 4 cannot hold 300 limbs
        # every shape gives the oracle's results
        g = W.rng(8)
        for R in (4, 8, 12, 16):
            x, y = W.class_operands(g, "max_pair", 33, 100)
            ctx.tune_set(dot.OP_MUL, 100, R)
            p = dot.mul(dev(x), dev(y), ctx=ctx)
            torch.cuda.synchronize()
            assert_same(host(p), oracle.mul(x, y), f"R={R}")
        for c in (1, 2, 4):
            x, y = W.class_operands(g, "runs", 3, 20000)
            ctx.tune_set(dot.OP_SUB, 20000, c)
            d, br = dot.sub(dev(x), dev(y), ctx=ctx)
            torch.cuda.synchronize()
            wd, wb = oracle.sub(x, y)
            assert_same(host(d), wd, f"chunks={c}")
            assert_same(host(br), wb, f"chunks={c}")
        assert ctx.check() == dot.OK
    finally:
        ctx.close()
