"""GPU multiply through the C ABI vs the CPU oracle, bit-exact."""
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
    p = D.mul(dev(x), dev(y))
    torch.cuda.synchronize()
    return host(p)


# every column shape: 4 / 8 / 12 / 16 columns per lane, with 1 to 8 ops per
# warp (e.g. 96: 12 columns, 4 ops; 150 and 160: 16 columns, 3 ops of 10
# lanes; 192: 12 columns, 2 ops)
SIZES = list(range(1, 41)) + [47, 63, 64, 65, 96, 100, 127, 128, 129, 150, 160, 192, 193, 200, 255, 256,
                              257, 300, 384, 385, 500, 511, 512]


@pytest.mark.parametrize("m", SIZES)
def test_sizes_and_classes(D, m):
    g = W.rng(2000 + m)
    for cls in W.CLASSES:
        x, y = W.class_operands(g, cls, 45, m)
        assert_same(run(D, x, y), oracle.mul(x, y), f"mul m={m} {cls}")


@pytest.mark.parametrize("m", [17, 20, 23, 24, 25, 28, 31, 32])
def test_one_product_per_thread_wide(D, m):
    """17..32 limbs in batches of at least 2^14 take one product per thread:
    every class, a ragged last block, and the scalar path of odd m."""
    assert D.plan(D.OP_MUL, m, (1 << 14) + 37).kernel == 4
    g = W.rng(2600 + m)
    for cls in W.CLASSES:
        x, y = W.class_operands(g, cls, (1 << 14) + 37, m)
        assert_same(run(D, x, y), oracle.mul(x, y, threads=8), f"m={m} {cls}")


def test_one_product_per_thread_unaligned(D):
    """The wide per-thread product on rows that are not 16-byte aligned (scalar
    loads and stores), with guard limbs around the output."""
    import torch
    m, n = 32, (1 << 14) + 5
    g = W.rng(2700)
    x, y = W.uniform_limbs(g, (n, m)), W.uniform_limbs(g, (n, m))
    xa = torch.zeros(n * m + 1, dtype=torch.int32, device="cuda")
    xa[1:] = dev(x).reshape(-1)
    out = torch.full((n * 2 * m + 2,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    view = out[1:1 + n * 2 * m].view(n, 2 * m)
    D.mul(xa[1:].view(n, m), dev(y), view)
    torch.cuda.synchronize()
    h = host(out)
    assert h[0] == 0x5A5A5A5A and h[-1] == 0x5A5A5A5A
    assert_same(h[1:1 + n * 2 * m].reshape(n, 2 * m), oracle.mul(x, y, threads=8), "unaligned")


def test_closed_form_all_ones(D):
    """(2^n - 1)^2 = 2^{2n} - 2^{n+1} + 1 for every supported size class."""
    for m in (1, 4, 8, 16, 17, 32, 256, 257, 512):
        x = np.full((3, m), 0xFFFFFFFF, np.uint32)
        p = run(D, x, x)
        want = np.zeros(2 * m, np.uint32)
        want[0] = 1
        if m == 1:
            want[1] = 0xFFFFFFFE
        else:
            want[m] = 0xFFFFFFFE
            want[m + 1:] = 0xFFFFFFFF
        assert_same(p, np.tile(want, (3, 1)), f"m={m}")


def test_correctness_mix(D):
    d = W.correctness_mix()
    assert_same(run(D, d["x"], d["y"]), oracle.mul(d["x"], d["y"], threads=8), "mix")


@pytest.mark.parametrize("m", W.BATCHED_MUL_SIZES)
def test_batched_mul_full(D, m):
    """The full 2^16-pair batched-multiply workload at each size."""
    x, y, _ = W.batched_mul(m)
    assert_same(run(D, x, y), oracle.mul(x, y, threads=16), f"batched m={m}")


def test_shared_operand_int32(D):
    f, b = W.shared_operand(batch=4096)
    a = np.tile(f, (b.shape[0], 1))
    assert_same(run(D, a, b), oracle.mul(a, b, threads=8), "shared")


def test_guard_bands(D):
    import torch
    g = W.rng(7)
    for m in (5, 32, 100, 256):
        x, y = W.class_operands(g, "uniform", 9, m)
        G = 64
        buf = torch.full((9 * 2 * m + 2 * G,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        out = buf[G:G + 18 * m].view(9, 2 * m)
        D.mul(dev(x), dev(y), out=out)
        torch.cuda.synchronize()
        hb = host(buf)
        assert (hb[:G] == 0x5A5A5A5A).all() and (hb[G + 18 * m:] == 0x5A5A5A5A).all()
        assert_same(hb[G:G + 18 * m].reshape(9, 2 * m), oracle.mul(x, y), f"m={m}")


def test_errors(D):
    import torch
    a = torch.zeros((2, 513), dtype=torch.int32, device="cuda")
    with pytest.raises(D.DotError) as e:
        D.mul(a, a)
    assert e.value.status == D.EUNSUPPORTED
    a = torch.zeros((2, 8), dtype=torch.int32, device="cuda")
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(D.DotError) as e:
        D.mul(buf[:16].view(2, 8), a, out=buf[8:40].view(2, 16))
    assert e.value.status == D.EINVAL


def test_ragged(D):
    import torch
    g = W.rng(41)
    sizes = [1, 2, 3, 4, 5, 8, 16, 17, 31, 32, 33, 64, 100, 129, 256, 257, 300, 383, 384, 385, 511, 512, 7, 0]
    a, b, off = W.ragged_uniform(g, sizes)
    want, poff = oracle.mul_ragged(a, b, off)
    out = torch.zeros(int(poff[-1]), dtype=torch.int32, device="cuda")
    D.mul_ragged(dev(a), dev(b), dev(off), dev(poff), out)
    torch.cuda.synchronize()
    assert D.default_context().check() == D.OK
    assert_same(host(out), want, "ragged mul")
    # an op above the size limit is skipped and reported
    a2, b2, off2 = W.ragged_uniform(g, [8, 600, 8])
    want2, poff2 = oracle.mul_ragged(a2, b2, off2)
    out2 = torch.zeros(int(poff2[-1]), dtype=torch.int32, device="cuda")
    D.mul_ragged(dev(a2), dev(b2), dev(off2), dev(poff2), out2)
    assert D.default_context().check() == D.EUNSUPPORTED
    h = host(out2)
    assert_same(h[:16], want2[:16], "before")
    assert_same(h[-16:], want2[-16:], "after")


def test_host_buffers(D):
    import torch
    g = W.rng(43)
    # (64, 150000): five 32 MB staging chunks, the last one partial, so both
    # staging buffers are reused
    for m, batch in ((32, 50000), (256, 3000), (13, 777), (64, 150000)):
        x, y = W.class_operands(g, "uniform", batch, m)
        xs = torch.from_numpy(x.view(np.int32)).pin_memory()
        ys = torch.from_numpy(y.view(np.int32)).pin_memory()
        out = torch.empty((batch, 2 * m), dtype=torch.int32).pin_memory()
        ctx = D.default_context()
        D.host_op(D.OP_MUL, xs.numpy(), ys.numpy(), out.numpy(), ctx=ctx)
        assert ctx.check() == D.OK
        assert_same(out.numpy().view(np.uint32), oracle.mul(x, y, threads=8), f"host mul m={m}")
