"""GPU add/sub through the C ABI vs the CPU oracle, bit-exact."""
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


def run(D, op, x, y):
    import torch
    a, b = dev(x), dev(y)
    s, c = (D.add if op == "add" else D.sub)(a, b)
    torch.cuda.synchronize()
    return host(s), host(c)


def want(op, x, y, threads=8):
    return (oracle.add if op == "add" else oracle.sub)(x, y, threads=threads)


SIZES = list(range(1, 41)) + [63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513,
                              1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097, 8191,
                              8192, 8193, 12289]


@pytest.mark.parametrize("op", ["add", "sub"])
@pytest.mark.parametrize("m", SIZES)
def test_sizes_and_classes(D, op, m):
    g = W.rng(1000 + m)
    for cls in W.CLASSES:
        batch = 3 if m > 2048 else 37
        x, y = W.class_operands(g, cls, batch, m)
        if op == "sub" and cls == "runs":
            x, y = W.sub_runs_operands(g, batch, m)
        s, c = run(D, op, x, y)
        ws, wc = want(op, x, y)
        assert_same(s, ws, f"{op} m={m} {cls}")
        assert_same(c, wc, f"{op} carry m={m} {cls}")


@pytest.mark.parametrize("op", ["add", "sub"])
def test_unaligned_scalar_path(D, op):
    """Odd m forces the 1-limb segment path (rows are not 16-byte aligned)."""
    g = W.rng(5)
    for m in (3, 7, 45, 130, 1001, 5003):
        x, y = W.class_operands(g, "runs", 9, m)
        s, c = run(D, op, x, y)
        ws, wc = want(op, x, y)
        assert_same(s, ws, f"{op} m={m}")
        assert_same(c, wc, f"{op} carry m={m}")


@pytest.mark.parametrize("op", ["add", "sub"])
def test_full_length_ripple_across_tiles(D, op):
    """(2^n - 1) + 1 and 0 - 1 at 2^22 bits: the carry crosses every tile."""
    m = 1 << 17
    x = np.full((2, m), 0xFFFFFFFF, np.uint32) if op == "add" else np.zeros((2, m), np.uint32)
    y = np.zeros((2, m), np.uint32)
    y[:, 0] = 1
    x[1, 5] = 0 if op == "add" else 7   # second row: the ripple stops early
    s, c = run(D, op, x, y)
    ws, wc = want(op, x, y)
    assert_same(s, ws, op)
    assert_same(c, wc, op + " carry")


@pytest.mark.parametrize("op", ["add", "sub"])
def test_long_operands_80_pairs(D, op):
    """80 pairs of 2^22-bit operands (84 MB of operands, 2560 tiles: more
    than one round of resident blocks, and a last round that not every block
    works on), with propagate runs crossing tiles and a full-length ripple
    row."""
    d = W.addsub_bandwidth(short_batch=0, long_batch=80)
    x, y = d[f"{op}_long"]
    s, c = run(D, op, x, y)
    ws, wc = want(op, x, y, threads=16)
    assert_same(s, ws, f"{op} long")
    assert_same(c, wc, f"{op} long carry")


@pytest.mark.parametrize("op", ["add", "sub"])
def test_long_operands_beside_another_kernel(D, op):
    """The long-operand kernel on its own context and stream while a large
    matmul holds SMs on another stream: not every block of the look-back
    kernel is resident at once, and its tiles still resolve in ticket order."""
    import torch
    g = W.rng(41)
    x, y = W.class_operands(g, "runs", 24, 1 << 17)
    ctx = D.Context(torch.cuda.current_device())
    try:
        busy = torch.cuda.Stream()
        mine = torch.cuda.Stream()
        m1 = torch.randn(8192, 8192, device="cuda")
        a, b = dev(x), dev(y)
        torch.cuda.synchronize()
        with torch.cuda.stream(busy):
            for _ in range(4):
                m1 = m1 @ m1.T
                m1 /= m1.abs().max()
        with torch.cuda.stream(mine):
            s, c = (D.add if op == "add" else D.sub)(a, b, ctx=ctx)
        torch.cuda.synchronize()
        assert ctx.check() == D.OK
        ws, wc = want(op, x, y, threads=16)
        assert_same(host(s), ws, f"{op} beside a matmul")
        assert_same(host(c), wc, f"{op} carry beside a matmul")
    finally:
        ctx.close()


def test_correctness_mix(D):
    d = W.correctness_mix()
    for op, (x, y) in (("add", (d["x"], d["y"])), ("sub", (d["a_sub"], d["b_sub"]))):
        s, c = run(D, op, x, y)
        ws, wc = want(op, x, y)
        assert_same(s, ws, op)
        assert_same(c, wc, op)
    # the sub operands satisfy a >= b: no borrow out
    assert not wc.any()


def test_addsub_bandwidth_full(D):
    """The full 2^20 x 4096-bit + 64 x 2^22-bit workload, every limb checked."""
    d = W.addsub_bandwidth()
    for name, (x, y) in d.items():
        op = name.split("_")[0]
        s, c = run(D, op, x, y)
        ws, wc = want(op, x, y, threads=16)
        assert_same(s, ws, name)
        assert_same(c, wc, name + " carry")


@pytest.mark.parametrize("op", ["add", "sub"])
def test_in_place_and_guard_bands(D, op):
    import torch
    g = W.rng(9)
    for m in (32, 128, 513, 4096 + 4):
        x, y = W.class_operands(g, "runs", 5, m)
        ws, wc = want(op, x, y)
        # result written over operand a
        a, b = dev(x), dev(y)
        fn = D.add if op == "add" else D.sub
        s, c = fn(a, b, out=a)
        torch.cuda.synchronize()
        assert_same(host(a), ws, f"in-place m={m}")
        assert_same(host(c), wc, f"in-place carry m={m}")
        # canary limbs around the output are untouched
        G = 64
        buf = torch.full((5 * m + 2 * G,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        cbuf = torch.full((5 + 2 * G,), 0x3C3C3C3C, dtype=torch.int32, device="cuda")
        out = buf[G:G + 5 * m].view(5, m)
        cout = cbuf[G:G + 5]
        fn(dev(x), dev(y), out, cout)
        torch.cuda.synchronize()
        hb, hc = host(buf), host(cbuf)
        assert (hb[:G] == 0x5A5A5A5A).all() and (hb[G + 5 * m:] == 0x5A5A5A5A).all()
        assert (hc[:G] == 0x3C3C3C3C).all() and (hc[G + 5:] == 0x3C3C3C3C).all()
        assert_same(hb[G:G + 5 * m].reshape(5, m), ws, "guarded")


def test_empty_and_invalid(D):
    import torch
    ctx = D.default_context()
    a = torch.zeros((4, 0), dtype=torch.int32, device="cuda")
    s, c = D.add(a, a)
    torch.cuda.synchronize()
    assert not host(c).any()
    z = torch.zeros((0, 8), dtype=torch.int32, device="cuda")
    D.add(z, z)
    # partial overlap of result and operand is rejected before any launch
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    x = buf[:32].view(4, 8)
    y = torch.zeros((4, 8), dtype=torch.int32, device="cuda")
    out = buf[4:36].view(4, 8)
    with pytest.raises(D.DotError) as e:
        D.add(x, y, out=out)
    assert e.value.status == D.EINVAL
    assert ctx.check() == D.OK


@pytest.mark.parametrize("op", ["add", "sub"])
def test_ragged(D, op):
    import torch
    g = W.rng(21)
    sizes = [0, 1, 2, 31, 32, 33, 100, 128, 129, 700, 4, 5000, 3]
    a, b, off = W.ragged_uniform(g, sizes, cls="runs")
    fn = D.add_ragged if op == "add" else D.sub_ragged
    s, c = fn(dev(a), dev(b), dev(off))
    torch.cuda.synchronize()
    ws, wc = (oracle.add_ragged if op == "add" else oracle.sub_ragged)(a, b, off)
    assert_same(host(s), ws, op)
    assert_same(host(c), wc, op + " carry")


def test_lookback_wait_is_bounded(D):
    """A tile that never publishes makes its successor's wait run out: the
    launch still ends, the status reads DOT_ETIMEOUT once, and the context
    keeps working (the failure is made on purpose through the debug hook)."""
    import torch
    ctx = D.Context(torch.cuda.current_device())
    try:
        ctx.set_wait_limit(20_000_000)   # 20 ms
        g = W.rng(3)
        m = 1 << 15
        x, y = W.class_operands(g, "ones", 2, m)   # every tile propagates
        ctx.debug_skip_publish(2)
        D.add(dev(x), dev(y), ctx=ctx)
        assert ctx.check() == D.ETIMEOUT
        assert ctx.check() == D.OK
        s, c = D.add(dev(x), dev(y), ctx=ctx)
        assert ctx.check() == D.OK
        ws, wc = oracle.add(x, y)
        assert_same(host(s), ws, "after timeout")
        assert_same(host(c), wc, "after timeout")
    finally:
        ctx.close()


@pytest.mark.parametrize("op", ["add", "sub"])
def test_host_buffers(D, op):
    import torch
    g = W.rng(31)
    for m, batch in ((128, 70000), (4096, 300), (7, 1000)):
        x, y = W.class_operands(g, "runs", batch, m)
        xs = torch.from_numpy(x.view(np.int32)).pin_memory()
        ys = torch.from_numpy(y.view(np.int32)).pin_memory()
        out = torch.empty_like(xs).pin_memory()
        car = torch.empty(batch, dtype=torch.int32).pin_memory()
        ctx = D.default_context()
        D.host_op(D.OP_ADD if op == "add" else D.OP_SUB, xs.numpy(), ys.numpy(), out.numpy(),
                  car.numpy(), ctx=ctx)
        assert ctx.check() == D.OK
        ws, wc = want(op, x, y)
        assert_same(out.numpy().view(np.uint32), ws, f"host {op} m={m}")
        assert_same(car.numpy().view(np.uint32), wc, f"host {op} carry m={m}")
