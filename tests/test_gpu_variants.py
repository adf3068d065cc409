"""mpn-style variants (carry-in, one-limb and shorter second operands) and the
batched square through the C ABI, bit-exact against the oracle."""
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


def sync():
    import torch
    torch.cuda.synchronize()


def _operands(seed, cls, batch, ma, mb):
    g = W.rng(seed)
    x, _ = W.class_operands(g, cls, batch, ma)
    _, y = W.class_operands(g, cls, batch, max(mb, 1))
    return x, np.ascontiguousarray(y[:, :mb]), g


@pytest.mark.parametrize("sub", [False, True])
@pytest.mark.parametrize("m", [1, 2, 31, 32, 33, 127, 128, 129, 1000, 5000])
@pytest.mark.parametrize("batch", [1, 7, 300])
def test_carry_in(D, sub, m, batch):
    x, y, g = _operands(3000 + m + batch, "runs", batch, m, m)
    cin = (g.integers(0, 2, batch) * g.integers(1, 5, batch)).astype(np.uint32)   # nonzero = 1
    fn = D.sub_nc if sub else D.add_nc
    s, c = fn(dev(x), dev(y), dev(cin))
    sync()
    ws, wc = (oracle.sub_gen if sub else oracle.add_gen)(x, y, cin)
    assert_same(host(s), ws, f"sub={sub} m={m}")
    assert_same(host(c), wc, "carry")


@pytest.mark.parametrize("sub", [False, True])
@pytest.mark.parametrize("cls", W.CLASSES)
def test_carry_in_value_classes(D, sub, cls):
    x, y, _ = _operands(3100, cls, 257, 64, 64)
    cin = np.ones(257, np.uint32)
    fn = D.sub_nc if sub else D.add_nc
    s, c = fn(dev(x), dev(y), dev(cin))
    sync()
    ws, wc = (oracle.sub_gen if sub else oracle.add_gen)(x, y, cin)
    assert_same(host(s), ws, cls)
    assert_same(host(c), wc, cls)


@pytest.mark.parametrize("sub", [False, True])
@pytest.mark.parametrize("m", [1, 2, 33, 200, 4097])
def test_one_limb(D, sub, m):
    x, y, _ = _operands(3200 + m, "uniform", 129, m, 1)
    # rows whose carry (borrow) ripples through every limb
    x[0] = 0xFFFFFFFF if not sub else 0
    y[0, 0] = 1
    fn = D.sub_1 if sub else D.add_1
    s, c = fn(dev(x), dev(np.ascontiguousarray(y[:, 0])))
    sync()
    ws, wc = (oracle.sub_gen if sub else oracle.add_gen)(x, y)
    assert_same(host(s), ws, f"m={m}")
    assert_same(host(c), wc, "carry")
    assert int(host(c)[0]) == 1


@pytest.mark.parametrize("sub", [False, True])
@pytest.mark.parametrize("ma,mb", [(1, 0), (1, 1), (5, 0), (5, 2), (64, 1), (64, 63), (64, 64),
                                   (300, 129), (2049, 2048)])
def test_unequal_lengths(D, sub, ma, mb):
    x, y, _ = _operands(3300 + ma + mb, "runs", 65, ma, mb)
    if ma > mb:
        # a tail that a carry (borrow) out of the common part must cross
        x[1, mb:] = 0xFFFFFFFF if not sub else 0
        if mb:
            x[1, :mb] = 0xFFFFFFFF if not sub else 0
            y[1, :mb] = 0
            y[1, 0] = 1
    fn = D.sub_unequal if sub else D.add_unequal
    s, c = fn(dev(x), dev(y) if mb else dev(np.zeros((65, 0), np.uint32)))
    sync()
    ws, wc = (oracle.sub_gen if sub else oracle.add_gen)(x, y)
    assert_same(host(s), ws, f"ma={ma} mb={mb}")
    assert_same(host(c), wc, "carry")


def test_in_place(D):
    x, y, g = _operands(3400, "uniform", 100, 40, 40)
    cin = g.integers(0, 2, 100).astype(np.uint32)
    a = dev(x)
    s, c = D.add_nc(a, dev(y), dev(cin), out=a)
    sync()
    ws, wc = oracle.add_gen(x, y, cin)
    assert_same(host(a), ws, "in place")
    assert_same(host(c), wc, "carry")


def test_variant_errors(D):
    import torch
    a = torch.zeros((4, 8), dtype=torch.int32, device="cuda")
    b = torch.zeros((4, 9), dtype=torch.int32, device="cuda")
    with pytest.raises(D.DotError) as e:
        D.add_unequal(a, b)   # mb > ma
    assert e.value.status == D.EINVAL
    out = torch.zeros((4, 8), dtype=torch.int32, device="cuda")
    carry = torch.zeros(4, dtype=torch.int32, device="cuda")
    ctx = D.default_context()
    st = D._stream(None)
    # carry-in pointer missing
    rc = D.lib().dot_add_nc(ctx.handle, D._ptr(a), D._ptr(a), D._vp(0), D._ptr(out), D._ptr(carry), 8, 4, st)
    assert rc == D.EINVAL
    # the output overlapping b (different strides)
    rc = D.lib().dot_add_unequal(ctx.handle, D._ptr(a), 8, D._ptr(out), 4, D._ptr(out), D._ptr(carry), 4, st)
    assert rc == D.EINVAL
    assert ctx.check() == D.OK


@pytest.mark.parametrize("m", [1, 2, 3, 4, 7, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 96, 100, 128, 150, 160,
                               192, 255, 256, 257, 300, 384, 385, 511, 512])
def test_square(D, m):
    g = W.rng(3500 + m)
    x, _ = W.class_operands(g, "uniform", 67, m)
    x[0] = 0xFFFFFFFF        # largest column sums: (X^m - 1)^2
    p = D.sqr(dev(x))
    sync()
    assert_same(host(p), oracle.sqr(x), f"m={m}")


@pytest.mark.parametrize("cls", W.CLASSES)
def test_square_value_classes(D, cls):
    g = W.rng(3600)
    x, _ = W.class_operands(g, cls, 129, 96)
    p = D.sqr(dev(x))
    q = D.mul(dev(x), dev(x))
    sync()
    assert_same(host(p), oracle.sqr(x), cls)
    assert_same(host(p), host(q), "square vs product")


def test_square_limits(D):
    import torch
    a = torch.zeros((2, 513), dtype=torch.int32, device="cuda")
    with pytest.raises(D.DotError) as e:
        D.sqr(a)
    assert e.value.status == D.EUNSUPPORTED
