"""Seeded synthetic workloads: shapes, determinism and structure (CPU only)."""
import numpy as np

from bigint import to_int
from paper_2604_21566_gb300 import workloads as W


def test_correctness_mix_structure():
    d = W.correctness_mix()
    x, y, a, b, cls = d["x"], d["y"], d["a_sub"], d["b_sub"], d["cls"]
    assert x.shape == y.shape == a.shape == b.shape == (4096, 32)
    assert x.dtype == np.uint32
    frac = np.bincount(cls, minlength=3) / cls.size
    assert abs(frac[0] - 0.5) < 0.03 and abs(frac[1] - 0.25) < 0.03
    ones = cls == 1
    assert (x[ones] == 0xFFFFFFFF).all() and not y[ones, 1:].any() and (y[ones, 0] > 0).all()
    # subtraction operands satisfy a >= b
    for k in range(0, 4096, 37):
        assert to_int(a[k]) >= to_int(b[k])
    # borrow dual in the all-ones class
    assert not a[ones, :-1].any() and (a[ones, -1] > 0).all()
    d2 = W.correctness_mix()
    assert (d2["x"] == x).all() and (d2["b_sub"] == b).all()


def test_addsub_bandwidth_small():
    d = W.addsub_bandwidth(short_batch=4096, short_m=128, long_batch=4, long_m=1 << 14,
                           long_runs=(256, 2048))
    xs, ys = d["add_short"]
    assert xs.shape == (4096, 128)
    run = (xs == 0xFFFFFFFF) & (ys == 0)
    assert 0.07 < run.mean() < 0.13
    xl, yl = d["add_long"]
    assert (xl[0] == 0xFFFFFFFF).all() and yl[0, 0] == 1 and not yl[0, 1:].any()
    sx, sy = d["sub_long"]
    assert not sx[0].any() and sy[0, 0] == 1


def test_batched_mul_and_ragged():
    x, y, maxed = W.batched_mul(8, batch=4096)
    assert x.shape == (4096, 8) and abs(maxed.mean() - 0.1) < 0.02
    assert (x[maxed] == 0xFFFFFFFF).all() and (y[maxed] == 0xFFFFFFFF).all()
    r = W.ragged_mixed(nops=5000)
    assert r["m"].min() >= 4 and r["m"].max() <= 512
    assert abs((r["op"] == W.OP_MUL).mean() - 0.4) < 1e-3
    assert int(r["a_off"][-1]) == r["a"].size == int(r["m"].sum())
    assert (r["r_len"] == np.where(r["op"] == W.OP_MUL, 2, 1) * r["m"]).all()
    for i in np.nonzero(r["op"] == W.OP_SUB)[0][:50]:
        lo, hi = int(r["a_off"][i]), int(r["a_off"][i + 1])
        assert to_int(r["a"][lo:hi]) >= to_int(r["b"][lo:hi])


def test_shared_operand():
    f, b = W.shared_operand(batch=128)
    assert f.shape == (64,) and b.shape == (128, 64)
