"""Guard bands: every entry point that writes device memory leaves the limbs
just before and after its outputs untouched, and still computes the oracle's
result.  Each output is a view into a larger buffer filled with a canary word;
the uneven sizes put the edges of the outputs inside warps and tiles."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, dev, host
from paper_2604_21566_gb300 import workloads as W

pytestmark = pytest.mark.gpu

G = 96                       # canary limbs on each side
CANARY = 0x5A5A5A5A
CANARY_C = 0x3C3C3C3C


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_21566_gb300 import dot
    dot.lib()
    return dot


class Guarded:
    """An output of `shape` inside a canary-filled buffer."""

    def __init__(self, shape, word=CANARY):
        import torch
        self.n = int(np.prod(shape))
        self.word = word
        self.buf = torch.full((self.n + 2 * G,), np.uint32(word).view(np.int32).item(), dtype=torch.int32,
                              device="cuda")
        self.view = self.buf[G:G + self.n].view(*shape)

    def check(self, what):
        import torch
        torch.cuda.synchronize()
        h = host(self.buf)
        assert (h[:G] == self.word).all(), f"{what}: wrote below its output"
        assert (h[G + self.n:] == self.word).all(), f"{what}: wrote past its output"
        return h[G:G + self.n]


def _pair(seed, batch, m, cls="runs"):
    g = W.rng(seed)
    return W.class_operands(g, cls, batch, m)


@pytest.mark.parametrize("m", [1, 3, 8, 33, 100, 257, 512])
def test_mul_and_sqr(D, m):
    x, y = _pair(6000 + m, 37, m)
    out = Guarded((37, 2 * m))
    D.mul(dev(x), dev(y), out.view)
    assert_same(out.check(f"mul m={m}").reshape(37, 2 * m), oracle.mul(x, y), f"mul m={m}")
    sq = Guarded((37, 2 * m))
    D.sqr(dev(x), sq.view)
    assert_same(sq.check(f"sqr m={m}").reshape(37, 2 * m), oracle.sqr(x), f"sqr m={m}")


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("m,batch", [(1, 5), (17, 129), (64, 300)])
def test_mul_shared(D, tc, m, batch):
    x, y = _pair(6100 + m, batch, m, "uniform")
    f = x[0]
    out = Guarded((batch, 2 * m))
    D.mul_shared(dev(f), dev(y), out.view, tensor_cores=tc)
    want = oracle.mul(np.ascontiguousarray(np.broadcast_to(f, y.shape)), y)
    assert_same(out.check(f"mul_shared tc={tc}").reshape(batch, 2 * m), want, f"tc={tc} m={m}")


@pytest.mark.parametrize("m", [513, 1031])
def test_mul_karatsuba(D, m):
    x, y = _pair(6200 + m, 5, m, "uniform")
    out = Guarded((5, 2 * m))
    D.mul_karatsuba(dev(x), dev(y), out.view)
    assert_same(out.check(f"karatsuba m={m}").reshape(5, 2 * m), oracle.mul(x, y, threads=8), f"m={m}")


@pytest.mark.parametrize("sub", [False, True])
@pytest.mark.parametrize("ma,mb", [(7, 7), (70, 1), (300, 129)])
def test_variants(D, sub, ma, mb):
    g = W.rng(6300 + ma + mb)
    x, _ = W.class_operands(g, "runs", 41, ma)
    _, y = W.class_operands(g, "runs", 41, mb)
    cin = g.integers(0, 2, 41).astype(np.uint32)
    out, car = Guarded((41, ma)), Guarded((41,), CANARY_C)
    if ma == mb:
        (D.sub_nc if sub else D.add_nc)(dev(x), dev(y), dev(cin), out.view, car.view)
        ws, wc = (oracle.sub_gen if sub else oracle.add_gen)(x, y, cin)
    elif mb == 1:
        (D.sub_1 if sub else D.add_1)(dev(x), dev(np.ascontiguousarray(y[:, 0])), out.view, car.view)
        ws, wc = (oracle.sub_gen if sub else oracle.add_gen)(x, y)
    else:
        (D.sub_unequal if sub else D.add_unequal)(dev(x), dev(y), out.view, car.view)
        ws, wc = (oracle.sub_gen if sub else oracle.add_gen)(x, y)
    assert_same(out.check("variant").reshape(41, ma), ws, f"sub={sub} ma={ma} mb={mb}")
    assert_same(car.check("variant carry"), wc, "carry")


def test_ragged(D):
    g = W.rng(6400)
    lens = np.array([1, 5, 32, 33, 130, 0, 7, 513], np.uint64)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    n = int(off[-1])
    x = g.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    y = g.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    out, car = Guarded((n,)), Guarded((lens.size,), CANARY_C)
    D.add_ragged(dev(x), dev(y), dev(off), out.view, car.view)
    ws, wc = oracle.add_ragged(x, y, off)
    assert_same(out.check("add_ragged"), ws, "add_ragged")
    assert_same(car.check("add_ragged carry"), wc, "carry")
    mlens = np.minimum(lens, 512)
    moff = np.concatenate([[0], np.cumsum(mlens)]).astype(np.uint64)
    poff = (2 * moff).astype(np.uint64)
    mx, my = x[:int(moff[-1])], y[:int(moff[-1])]
    prod = Guarded((int(poff[-1]),))
    D.mul_ragged(dev(mx), dev(my), dev(moff), dev(poff), prod.view)
    wp, _ = oracle.mul_ragged(mx, my, moff)
    assert_same(prod.check("mul_ragged"), wp, "mul_ragged")
