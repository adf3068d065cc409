"""Batched Karatsuba above the base case through the C ABI, bit-exact against
the oracle's row-wise schoolbook product."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, dev, host
from paper_2604_21566_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_21566_gb300 import dot
    dot.lib()
    return dot


def run(D, x, y):
    import torch
    p = D.mul_karatsuba(dev(x), dev(y))
    torch.cuda.synchronize()
    return host(p)


@pytest.mark.parametrize("m", [1, 100, 384, 385, 512, 513, 514, 600, 1023, 1024, 1025, 2048, 3001, 4096])
def test_sizes(D, m):
    g = W.rng(4000 + m)
    batch = 9 if m <= 1025 else 4
    x, y = W.class_operands(g, "uniform", batch, m)
    x[0] = y[0] = 0xFFFFFFFF          # (X^m - 1)^2
    assert_same(run(D, x, y), oracle.mul(x, y, threads=8), f"m={m}")


@pytest.mark.parametrize("cls", W.CLASSES)
def test_value_classes(D, cls):
    """Halves that are equal, ordered either way, or zero: every sign case of
    |A_H - A_L| and |B_H - B_L|."""
    g = W.rng(4100)
    x, y = W.class_operands(g, cls, 16, 1100)
    # rows whose halves compare equal, or differ only in the lowest limb
    x[1, 550:] = x[1, :550]
    y[1, 550:] = y[1, :550]
    x[2, 550:] = x[2, :550]
    x[2, 0] ^= 1
    y[3, :550] = y[3, 550:]
    assert_same(run(D, x, y), oracle.mul(x, y, threads=8), cls)


def test_several_levels(D):
    """16384 limbs: six halvings down to 256-limb base cases (3^6 = 729
    base products per operation)."""
    g = W.rng(4200)
    x, y = W.class_operands(g, "uniform", 2, 16384)
    assert_same(run(D, x, y), oracle.mul(x, y, threads=8), "m=16384")


def test_base_case_is_dot_mul(D):
    import torch
    g = W.rng(4300)
    x, y = W.class_operands(g, "runs", 300, 257)
    p = D.mul_karatsuba(dev(x), dev(y))
    q = D.mul(dev(x), dev(y))
    torch.cuda.synchronize()
    assert_same(host(p), host(q), "m=257")


def test_limits(D):
    import torch
    ctx = D.default_context()
    a = torch.zeros((2, 8), dtype=torch.int32, device="cuda")
    p = torch.zeros((2, 16), dtype=torch.int32, device="cuda")
    st = D._stream(None)
    # more limbs than the workspace plan allows
    rc = D.lib().dot_mul_karatsuba(ctx.handle, D._ptr(a), D._ptr(a), D._ptr(p), (1 << 20) + 1, 1, st)
    assert rc == D.EINVAL
    # output overlapping an operand
    rc = D.lib().dot_mul_karatsuba(ctx.handle, D._ptr(p), D._ptr(a), D._ptr(p), 8, 2, st)
    assert rc == D.EINVAL
    assert ctx.check() == D.OK
