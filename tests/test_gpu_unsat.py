"""dot_mul_unsat (products of 27-bit-digit operands, the unsaturated radix of
Sec. 2.1) through the C ABI vs the CPU oracle's radix-2^27 schoolbook,
bit-exact."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, dev, host
from paper_2604_21566_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BITS = W.UNSAT_BITS
CLASSES = ("uniform", "max_pair", "zeros", "sparse", "ones")


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_21566_gb300 import dot
    dot.lib()
    return dot


def run(D, x, y, ctx=None):
    import torch
    p = D.mul_unsat(dev(x), dev(y), ctx=ctx)
    torch.cuda.synchronize()
    return host(p)


# every column-block shape (4 / 8 / 12 / 16 digits per lane) and run width,
# tile edges and the largest size
SIZES = list(range(1, 41)) + [63, 64, 65, 96, 127, 128, 129, 150, 152, 192, 193, 256, 257, 300, 304,
                              384, 385, 500, 511, 512]


@pytest.mark.parametrize("n", SIZES)
def test_sizes_and_classes(D, n):
    g = W.rng(3000 + n)
    for cls in CLASSES:
        x, y = W.radix_operands(g, cls, 37, n, BITS)
        assert_same(run(D, x, y), oracle.mul_radix(x, y, BITS), f"unsat n={n} {cls}")


def test_closed_form_all_max(D):
    """(2^(27n) - 1)^2: digits 1, 0.., 2^27 - 2, 2^27 - 1 .. -- the largest
    column sums every block shape sees."""
    top = (1 << BITS) - 1
    for n in (1, 4, 16, 17, 64, 152, 304, 512):
        x = np.full((5, n), top, np.uint32)
        want = np.zeros(2 * n, np.uint32)
        want[0] = 1
        want[n] = top - 1
        want[n + 1:] = top
        if n == 1:
            want = np.array([1, top - 1], np.uint32)
        assert_same(run(D, x, x), np.tile(want, (5, 1)), f"n={n}")


@pytest.mark.parametrize("bits_total", [256, 1024, 4096, 8192])
def test_workload_full(D, bits_total):
    """2^16 pairs at the batched-multiply workload's sizes (10, 38, 152 and
    304 digits), every row checked."""
    x, y = W.unsaturated_mul(bits_total)
    assert_same(run(D, x, y), oracle.mul_radix(x, y, BITS, threads=16), f"workload {bits_total} bits")


def test_same_integer_as_the_saturated_product(D):
    """The same integers multiplied in radix 2^27 and in radix 2^32 (dot_mul)
    give the same product: pins the digit layout against the limb layout."""
    import torch
    from bigint import from_int, from_int_radix, to_int, to_int_radix
    g = W.rng(44)
    x27, y27 = W.radix_operands(g, "uniform", 16, 76, BITS)   # 2052 bits
    xs = np.stack([from_int(to_int_radix(r, BITS), 65) for r in x27])
    ys = np.stack([from_int(to_int_radix(r, BITS), 65) for r in y27])
    p27 = run(D, x27, y27)
    p32 = host(D.mul(dev(xs), dev(ys)))
    torch.cuda.synchronize()
    for k in range(16):
        assert to_int_radix(p27[k], BITS) == to_int(p32[k])


def test_bad_digit_recorded_and_limits(D):
    import torch
    ctx = D.Context(0)
    try:
        x = np.zeros((4, 8), np.uint32)
        x[2, 3] = 1 << BITS                # not a 27-bit digit
        D.mul_unsat(dev(x), dev(x), ctx=ctx)
        assert ctx.check() == D.EINVAL
        assert ctx.check() == D.OK         # the status is cleared by the check
        big = torch.zeros((2, D.UNSAT_MAX_DIGITS + 1), dtype=torch.int32, device="cuda")
        with pytest.raises(D.DotError) as e:
            D.mul_unsat(big, big, ctx=ctx)
        assert e.value.status == D.EUNSUPPORTED
        # guard bands around the output stay untouched
        g = W.rng(5)
        x, y = W.radix_operands(g, "uniform", 9, 37, BITS)
        out = torch.full((9 * 74 + 64,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        view = out[32:32 + 9 * 74].view(9, 74)
        D.mul_unsat(dev(x), dev(y), out=view, ctx=ctx)
        torch.cuda.synchronize()
        h = host(out)
        assert (h[:32] == 0x5A5A5A5A).all() and (h[-32:] == 0x5A5A5A5A).all()
        assert_same(h[32:32 + 9 * 74].reshape(9, 74), oracle.mul_radix(x, y, BITS), "guarded")
        assert ctx.check() == D.OK
    finally:
        ctx.close()
