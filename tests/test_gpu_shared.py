"""Shared-operand products (one fixed operand x a batch) through the C ABI:
the tensor-core Toeplitz path and the INT32 path, bit-exact vs the oracle.
Up to 64 limbs the tensor path sums each column in one K slice of 256 digits;
from 65 to 128 limbs in two slices whose sums are added before the carry pass."""
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


def run(D, f, b, tc):
    import torch
    p = D.mul_shared(dev(f), dev(b), tensor_cores=tc)
    torch.cuda.synchronize()
    return host(p)


def want(f, b):
    return oracle.mul(np.ascontiguousarray(np.broadcast_to(f, b.shape)), b, threads=8)


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("m", [1, 2, 3, 7, 8, 16, 17, 31, 32, 33, 48, 63, 64, 65, 66, 80, 95, 96, 97, 127, 128])
@pytest.mark.parametrize("batch", [1, 127, 128, 129, 1000])
def test_sizes(D, tc, m, batch):
    g = W.rng(5000 + 13 * m + batch)
    f = W.uniform_limbs(g, m)
    b = W.uniform_limbs(g, (batch, m))
    assert_same(run(D, f, b, tc), want(f, b), f"tc={tc} m={m} batch={batch}")


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("m", [64, 65, 128])
def test_largest_column_sums(D, tc, m):
    """All-ones digits everywhere: every column sum of a K slice reaches its
    bound 256 * 255^2 = 16,646,400 (just under 2^24); the result is
    (2^n - 1)^2."""
    f = np.full(m, 0xFFFFFFFF, np.uint32)
    b = np.full((300, m), 0xFFFFFFFF, np.uint32)
    p = run(D, f, b, tc)
    wantrow = np.zeros(2 * m, np.uint32)
    wantrow[0] = 1
    wantrow[m] = 0xFFFFFFFE
    wantrow[m + 1:] = 0xFFFFFFFF
    assert_same(p, np.tile(wantrow, (300, 1)), f"tc={tc}")


FIXED_PATTERNS = {
    "bytes_0x80": 0x80808080,      # balanced digits -128, then -127 each
    "bytes_0x7f": 0x7F7F7F7F,
    "alt_7f_80": 0x807F807F,       # balanced digits alternate near +-128
    "alt_80_7f": 0x7F807F80,
    "all_ones": 0xFFFFFFFF,        # every digit -1 with a carry, top digit +1
    "top_bit": 0x80000000,
}


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("pattern", sorted(FIXED_PATTERNS))
@pytest.mark.parametrize("m", [1, 5, 64, 65, 100, 128])
def test_digit_extremes(D, tc, pattern, m):
    """Fixed operands whose balanced digits sit at +-128 and batch rows of all
    zero digits (shifted to -128) or all 0xFF digits (127): the raw column sums
    reach the ends of their range, and zero rows must give exact zeros."""
    g = W.rng(900 + m)
    f = np.full(m, FIXED_PATTERNS[pattern], np.uint32)
    rows = [np.zeros(m, np.uint32), np.full(m, 0xFFFFFFFF, np.uint32), np.full(m, 0x80808080, np.uint32),
            np.full(m, 0x7F7F7F7F, np.uint32)]
    b = np.vstack(rows + [W.uniform_limbs(g, (200, m))])
    assert_same(run(D, f, b, tc), want(f, b), f"{pattern} m={m} tc={tc}")


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("m", [64, 128])
def test_value_classes(D, tc, m):
    g = W.rng(77 + m)
    for cls in W.CLASSES:
        x, y = W.class_operands(g, cls, 257, m)
        f = x[0]
        assert_same(run(D, f, y, tc), want(f, y), f"{cls} m={m} tc={tc}")


def test_shared_operand_workload_full(D):
    """The 2^16-operand, 2048-bit workload: tensor-core and INT32 paths agree
    with each other on every row and with the oracle on every row."""
    f, b = W.shared_operand()
    p_tc = run(D, f, b, True)
    p_int = run(D, f, b, False)
    assert_same(p_tc, p_int, "tensor vs int32")
    assert_same(p_tc, want(f, b), "tensor vs oracle")


@pytest.mark.parametrize("m", [96, 128])
def test_split_k_workload(D, m):
    """2^16 operands at 3072 and 4096 bits (two K slices): every row against
    the oracle."""
    f, b = W.shared_operand(m=m)
    assert_same(run(D, f, b, True), want(f, b), f"tensor m={m}")


def test_rows_past_batch_and_unaligned_output(D):
    """An odd m (no tensor store: rows are written with plain stores) and an
    output offset by one limb: guard limbs around it stay untouched."""
    import torch
    g = W.rng(31)
    for m in (33, 65, 127):
        f = W.uniform_limbs(g, m)
        b = W.uniform_limbs(g, (300, m))
        out = torch.full((300 * 2 * m + 2,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        view = out[1:1 + 300 * 2 * m].view(300, 2 * m)
        D.mul_shared(dev(f), dev(b), out=view, tensor_cores=True)
        torch.cuda.synchronize()
        h = host(out)
        assert h[0] == 0x5A5A5A5A and h[-1] == 0x5A5A5A5A, m
        assert_same(h[1:1 + 300 * 2 * m].reshape(300, 2 * m), want(f, b), f"unaligned m={m}")


def test_limits(D):
    import torch
    f = torch.zeros(129, dtype=torch.int32, device="cuda")
    b = torch.zeros((4, 129), dtype=torch.int32, device="cuda")
    with pytest.raises(D.DotError) as e:
        D.mul_shared(f, b, tensor_cores=True)
    assert e.value.status == D.EUNSUPPORTED
    D.mul_shared(f, b, tensor_cores=False)   # the INT32 path takes it
    assert D.default_context().check() == D.OK
