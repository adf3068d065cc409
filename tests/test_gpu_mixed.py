"""Mixed ragged batches (bucketed persistent kernel from a captured graph)
through the C ABI vs the CPU oracle, bit-exact."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, dev, host
from paper_2604_21566_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DESC = np.dtype([("op", "<u4"), ("m", "<u4"), ("a_off", "<u8"), ("b_off", "<u8"), ("r_off", "<u8")])


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_21566_gb300 import dot
    dot.lib()
    return dot


def descriptors(op, m, a_off, r_off):
    d = np.zeros(len(op), dtype=DESC)
    d["op"] = op
    d["m"] = m
    d["a_off"] = a_off
    d["b_off"] = a_off
    d["r_off"] = r_off
    return d


def run_mixed(D, ctx, d, a, b, r_len):
    import torch
    desc = torch.from_numpy(d.view(np.uint8).copy()).cuda()
    r = torch.zeros(int(r_len), dtype=torch.int32, device="cuda")
    carry = torch.full((len(d),), 7, dtype=torch.int32, device="cuda")
    D.mixed_ragged(desc, dev(a), dev(b), r, carry, ctx=ctx)
    st = ctx.check()
    return host(r), host(carry), st


def want_mixed(d, a, b, r_len):
    return oracle.mixed(d["op"], d["m"], d["a_off"], d["b_off"], d["r_off"], a, b, r_len)


def test_ragged_mixed_workload_full(D):
    """The 200k-op mixed workload (30% add, 30% sub, 40% mul, 128..16384 bits)."""
    w = W.ragged_mixed()
    d = descriptors(w["op"], w["m"], w["a_off"][:-1], w["r_off"][:-1])
    ctx = D.Context()
    try:
        r, c, st = run_mixed(D, ctx, d, w["a"], w["b"], w["r_off"][-1])
        assert st == D.OK
        wr, wc = want_mixed(d, w["a"], w["b"], w["r_off"][-1])
        assert_same(c, wc, "carries")
        assert_same(r, wr, "results")
        # the captured graph is replayed: same answer the second time
        r2, c2, st = run_mixed(D, ctx, d, w["a"], w["b"], w["r_off"][-1])
        assert st == D.OK
        assert_same(r2, wr, "replay")
        assert_same(c2, wc, "replay carries")
    finally:
        ctx.close()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_small_batches_every_bucket(D, seed):
    """Every size class incl. the boundaries between buckets, several calls
    of different lengths on one context (graph parameters updated per call)."""
    g = W.rng(300 + seed)
    sizes = [1, 2, 3, 4, 15, 16, 17, 63, 64, 65, 127, 128, 129, 255, 256, 257, 383, 384, 385, 511, 512,
             700, 1000, 5]
    n = 3 * len(sizes)
    op = np.array([k % 3 for k in range(n)], dtype=np.uint32)
    g.shuffle(op)
    m = np.array((sizes * 3)[:n], dtype=np.int64)
    g.shuffle(m)
    m[(op == 2) & (m > 512)] = 512
    a, b, off = W.ragged_uniform(g, m, cls="runs")
    r_len = np.where(op == 2, 2 * m, m)
    r_off = np.concatenate([[0], np.cumsum(r_len)]).astype(np.uint64)
    d = descriptors(op, m, off[:-1], r_off[:-1])
    ctx = D.default_context()
    for k in (n, n // 2, 7, n):
        dk = d[:k]
        r, c, st = run_mixed(D, ctx, dk, a, b, r_off[-1])
        assert st == D.OK
        wr, wc = want_mixed(dk, a, b, r_off[-1])
        assert_same(c, wc, f"carries k={k}")
        assert_same(r, wr, f"results k={k}")


@pytest.mark.parametrize("cls", ["uniform", "runs", "ones", "max_pair"])
def test_every_product_size(D, cls):
    """One multiply of every size from 1 to 512 limbs, so that every bucket,
    every boundary between buckets and every columns-per-lane shape (R = 4 to
    16, odd R included) runs, twice over: once from operands packed back to
    back (most rows not 16-byte aligned) and once with every row padded to a
    multiple of 4 limbs; a few add/sub ops ride along."""
    g = W.rng(800 + W.CLASSES.index(cls))
    for padded in (False, True):
        m = np.arange(1, 513, dtype=np.int64)
        op = np.full(m.size, 2, dtype=np.uint32)
        m = np.concatenate([m, [5, 300, 130]])
        op = np.concatenate([op, np.array([0, 1, 0], dtype=np.uint32)])
        if padded:
            stored = (m + 3) // 4 * 4
            a0, b0, off0 = W.ragged_uniform(g, stored, cls=cls)
            # zero the padding: only the first m limbs of each row are operands
            a, b = a0.copy(), b0.copy()
            for k in range(m.size):
                a[int(off0[k]) + int(m[k]):int(off0[k + 1])] = 0
                b[int(off0[k]) + int(m[k]):int(off0[k + 1])] = 0
            off = off0
        else:
            a, b, off = W.ragged_uniform(g, m, cls=cls)
        r_len = np.where(op == 2, 2 * m, m)
        r_len = (r_len + 3) // 4 * 4 if padded else r_len
        r_off = np.concatenate([[0], np.cumsum(r_len)]).astype(np.uint64)
        d = descriptors(op, m, off[:-1], r_off[:-1])
        ctx = D.default_context()
        r, c, st = run_mixed(D, ctx, d, a, b, r_off[-1])
        assert st == D.OK
        wr, wc = want_mixed(d, a, b, r_off[-1])
        assert_same(c, wc, f"carries {cls} padded={padded}")
        assert_same(r, wr, f"results {cls} padded={padded}")


def test_bad_descriptors_reported(D):
    g = W.rng(9)
    sizes = np.array([8, 600, 8, 5, 0], dtype=np.int64)
    op = np.array([2, 2, 9, 0, 1], dtype=np.uint32)   # mul too long, unknown op, empty op
    a, b, off = W.ragged_uniform(g, sizes)
    r_len = np.where(op == 2, 2 * sizes, sizes)
    r_off = np.concatenate([[0], np.cumsum(r_len)]).astype(np.uint64)
    d = descriptors(op, sizes, off[:-1], r_off[:-1])
    ctx = D.default_context()
    r, c, st = run_mixed(D, ctx, d, a, b, r_off[-1])
    assert st in (D.EUNSUPPORTED, D.EINVAL)
    ok = np.array([0, 3])
    wr, wc = want_mixed(d[ok], a, b, r_off[-1])
    assert_same(r[:16], wr[:16], "valid mul")
    lo = int(r_off[3])
    assert_same(r[lo:lo + 5], wr[lo:lo + 5], "valid add")
    assert c[1] == 0 and c[2] == 0 and c[4] == 0
