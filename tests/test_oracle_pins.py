"""Pins of the CPU oracle against things other than itself (CPU only).

* Python's own big integers (an independent arbitrary-precision implementation)
  for random operands of every value class, m up to 512 limbs;
* brute force on <= 64-bit operands (m = 1, 2) over an edge-value set;
* closed forms: (2^n - 1) + 1 = 2^n, 0 - 1 = 2^n - 1 with borrow,
  (2^n - 1)^2 = 2^{2n} - 2^{n+1} + 1;
* invariants: (a + b) - b = a, a - a = 0, a + b = b + a, ab = ba,
  a (b + c) = ab + ac, a * 1 = a, a * 0 = 0, a * X^j = shift;
* the m = 5 worked example of Sec. 3.2, tests/golden;
* the mpn-style variants (carry-in, zero-padded shorter operand) and the
  square, against Python's integers and closed forms;
* the carry-probability lemma of the appendix (Pr[carry] = 1/2 - 2^-(k+1)).

Each pin is a plain function so that tests/test_oracle_mutants.py can rerun it
against deliberately broken copies of the oracle.
"""
import os

import numpy as np
import pytest

import oracle
from bigint import X, from_int, from_int_radix, rows_to_ints, to_int, to_int_radix
from paper_2604_21566_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EDGE = [0, 1, 2, 1 << 31, (1 << 32) - 2, (1 << 32) - 1]


# ---------------------------------------------------------------- pins ----
def pin_python_int_addsub():
    g = W.rng(11)
    for m in (1, 2, 3, 7, 32, 33, 128, 257, 512):
        for cls in W.CLASSES:
            x, y = W.class_operands(g, cls, 6, m)
            s, c = oracle.add(x, y)
            d, br = oracle.sub(x, y)
            for k in range(x.shape[0]):
                A, B = to_int(x[k]), to_int(y[k])
                assert to_int(s[k]) + int(c[k]) * X ** m == A + B, (m, cls, k)
                assert int(c[k]) in (0, 1)
                assert to_int(d[k]) - int(br[k]) * X ** m == A - B, (m, cls, k)
                assert int(br[k]) in (0, 1)


def pin_python_int_mul():
    g = W.rng(12)
    for m in (1, 2, 3, 5, 8, 31, 64, 129):
        for cls in W.CLASSES:
            x, y = W.class_operands(g, cls, 4, m)
            p = oracle.mul(x, y)
            assert p.shape == (x.shape[0], 2 * m)
            for k in range(x.shape[0]):
                assert to_int(p[k]) == to_int(x[k]) * to_int(y[k]), (m, cls, k)


def pin_python_int_mul_columns():
    g = W.rng(13)
    for m in (1, 2, 3, 4, 5, 8, 17, 64):
        for cls in ("uniform", "max_pair", "ones", "sparse"):
            x, y = W.class_operands(g, cls, 4, m)
            p = oracle.mul_columns(x, y)
            for k in range(x.shape[0]):
                assert to_int(p[k]) == to_int(x[k]) * to_int(y[k]), (m, cls, k)


def pin_brute_force_small():
    """Every pair over the edge set for m = 1 and m = 2 (<= 64-bit values)."""
    vals1 = np.array(EDGE, dtype=np.uint32)[:, None]
    vals2 = np.array([[u, v] for u in EDGE for v in EDGE], dtype=np.uint32)
    for vals in (vals1, vals2):
        m = vals.shape[1]
        n = vals.shape[0]
        x = np.repeat(vals, n, axis=0)
        y = np.tile(vals, (n, 1))
        s, c = oracle.add(x, y)
        d, br = oracle.sub(x, y)
        p = oracle.mul(x, y)
        A = rows_to_ints(x)
        B = rows_to_ints(y)
        for k in range(x.shape[0]):
            tot = A[k] + B[k]
            assert to_int(s[k]) == tot % X ** m and int(c[k]) == tot >> (32 * m)
            dif = A[k] - B[k]
            assert to_int(d[k]) == dif % X ** m and int(br[k]) == (1 if dif < 0 else 0)
            assert to_int(p[k]) == A[k] * B[k]


def pin_closed_forms():
    for m in (1, 2, 5, 32, 128):
        ones = np.full((1, m), 0xFFFFFFFF, dtype=np.uint32)
        one = np.zeros((1, m), dtype=np.uint32)
        one[0, 0] = 1
        zero = np.zeros((1, m), dtype=np.uint32)
        # (2^n - 1) + 1 = 2^n: all-zero limbs and carry 1
        s, c = oracle.add(ones, one)
        assert not s.any() and c[0] == 1
        s, c = oracle.add(one, ones)
        assert not s.any() and c[0] == 1
        # 0 - 1 = 2^n - 1 with borrow 1
        d, br = oracle.sub(zero, one)
        assert (d == 0xFFFFFFFF).all() and br[0] == 1
        # (2^n - 1)^2 = 2^{2n} - 2^{n+1} + 1: limbs [1, 0.., 2^32-2, 2^32-1 ..]
        want = np.zeros(2 * m, dtype=np.uint32)
        want[0] = 1
        want[m] = 0xFFFFFFFE
        want[m + 1:] = 0xFFFFFFFF
        if m == 1:
            want = np.array([1, 0xFFFFFFFE], dtype=np.uint32)
        assert (oracle.mul(ones, ones)[0] == want).all(), m
        assert (oracle.mul_columns(ones, ones)[0] == want).all(), m


def pin_invariants():
    g = W.rng(14)
    for m in (1, 3, 16, 100):
        a, b = W.class_operands(g, "uniform", 8, m)
        c_, _ = W.class_operands(g, "uniform", 8, m)
        # (a + b) - b = a, borrow equals the carry
        s, cy = oracle.add(a, b)
        d, br = oracle.sub(s, b)
        assert (d == a).all() and (br == cy).all()
        # a - a = 0, borrow 0 ; a + b = b + a
        d, br = oracle.sub(a, a)
        assert not d.any() and not br.any()
        s2, cy2 = oracle.add(b, a)
        assert (s2 == s).all() and (cy2 == cy).all()
        # ab = ba
        assert (oracle.mul(a, b) == oracle.mul(b, a)).all()
        # a (b + c) = ab + ac, with b + c taken as m+1 limbs
        bc, cbc = oracle.add(b, c_)
        bc1 = np.concatenate([bc, cbc[:, None]], axis=1)
        a1 = np.concatenate([a, np.zeros((a.shape[0], 1), np.uint32)], axis=1)
        lhs = oracle.mul(a1, bc1)                     # 2m + 2 limbs
        rsum, rcar = oracle.add(oracle.mul(a, b), oracle.mul(a, c_))   # 2m limbs + carry
        assert (lhs[:, :2 * m] == rsum).all()
        assert (lhs[:, 2 * m] == rcar).all() and not lhs[:, 2 * m + 1].any()
        # a * 1 = a, a * 0 = 0, a * X^j = a shifted by j limbs
        one = np.zeros_like(a)
        one[:, 0] = 1
        p = oracle.mul(a, one)
        assert (p[:, :m] == a).all() and not p[:, m:].any()
        assert not oracle.mul(a, np.zeros_like(a)).any()
        for j in range(m):
            xj = np.zeros_like(a)
            xj[:, j] = 1
            p = oracle.mul(a, xj)
            assert (p[:, j:j + m] == a).all() and not p[:, :j].any() and not p[:, j + m:].any()


def pin_column_worked_example():
    """The m = 5 walkthrough of Sec. 3.2 (column pair counts, the pairs of
    column 4 in order, 25 pairs, where pair (2, 3) lands), values from
    tests/golden."""
    gold = {}
    with open(os.path.join(GOLDEN, "column_pairs_m5_worked_example.txt")) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                k, *v = ln.split()
                gold[k] = v
    m = 5
    ia, jb, nc = oracle.column_pairs(m)
    assert nc.size == int(gold["columns"][0])
    assert list(nc) == [int(t) for t in gold["pairs_per_column"]]
    # num_pairs = min(c+1, m, 2m-1-c) is the same count
    assert list(nc) == [min(c + 1, m, 2 * m - 1 - c) for c in range(2 * m - 1)]
    start4 = int(nc[:4].sum())
    got4 = [f"{i},{j}" for i, j in zip(ia[start4:start4 + nc[4]], jb[start4:start4 + nc[4]])]
    assert got4 == gold["column4_pairs"]
    assert ia.size == int(gold["gathered_entries"][0])
    full, rem = divmod(ia.size, 8)
    assert [full, rem] == [int(t) for t in gold["phase2_chunks_w8"]]
    # pair (2,3) sits in column 5's group, so its low half goes to column 5
    # and its high half to column 6 (Phase 3)
    t = [k for k in range(ia.size) if ia[k] == 2 and jb[k] == 3][0]
    col = int(np.searchsorted(np.cumsum(nc), t, side="right"))
    assert [col, col + 1] == [int(t) for t in gold["pair_2_3_columns"]]
    # the low and high halves of that single product land in columns 5 and 6
    a = np.zeros((1, m), np.uint32)
    b = np.zeros((1, m), np.uint32)
    a[0, 2] = 0x89ABCDEF
    b[0, 3] = 0xFEDCBA98
    p = oracle.mul_columns(a, b)
    prod = 0x89ABCDEF * 0xFEDCBA98
    want = np.zeros(2 * m, np.uint32)
    want[5] = prod & 0xFFFFFFFF
    want[6] = prod >> 32
    assert (p[0] == want).all()
    assert p.shape[1] == int(gold["product_limbs"][0])


def pin_ragged_and_mixed():
    g = W.rng(15)
    sizes = [0, 1, 5, 32, 3, 0, 130, 7]
    a, b, off = W.ragged_uniform(g, sizes)
    s, c = oracle.add_ragged(a, b, off)
    d, br = oracle.sub_ragged(a, b, off)
    p, poff = oracle.mul_ragged(a, b, off)
    for k, mk in enumerate(sizes):
        lo, hi = int(off[k]), int(off[k + 1])
        A, B = to_int(a[lo:hi]), to_int(b[lo:hi])
        assert to_int(s[lo:hi]) + int(c[k]) * X ** mk == A + B
        assert to_int(d[lo:hi]) - int(br[k]) * X ** mk == A - B
        assert to_int(p[int(poff[k]):int(poff[k + 1])]) == A * B
    # mixed descriptors
    op = np.array([0, 1, 2, 2, 0, 1, 2, 0], dtype=np.uint32)
    r_len = np.where(op == 2, 2, 1) * np.array(sizes)
    r_off = np.concatenate([[0], np.cumsum(r_len)]).astype(np.uint64)
    m32 = np.array(sizes, dtype=np.uint32)
    r, cc = oracle.mixed(op, m32, off[:-1], off[:-1], r_off[:-1], a, b, r_off[-1])
    for k, mk in enumerate(sizes):
        lo, hi = int(off[k]), int(off[k + 1])
        A, B = to_int(a[lo:hi]), to_int(b[lo:hi])
        R = to_int(r[int(r_off[k]):int(r_off[k]) + int(r_len[k])])
        if op[k] == 0:
            assert R + int(cc[k]) * X ** mk == A + B
        elif op[k] == 1:
            assert R - int(cc[k]) * X ** mk == A - B
        else:
            assert R == A * B and cc[k] == 0


def pin_carry_probability():
    """Appendix lemma: for uniform k-bit limbs Pr[X + Y >= 2^k] = 1/2 - 2^-(k+1).
    1-limb additions of 2^20 uniform pairs: the carry rate lies within 5 sigma."""
    g = W.rng(16)
    n = 1 << 20
    x, y = W.class_operands(g, "uniform", n, 1)
    _, c = oracle.add(x, y)
    p = 0.5 - 2.0 ** -33
    sigma = (p * (1 - p) / n) ** 0.5
    assert abs(c.mean() - p) < 5 * sigma
    # and the carry is exactly the lemma's condition on the low word: s < x
    s, _ = oracle.add(x, y)
    assert ((s[:, 0] < x[:, 0]).astype(np.uint32) == c).all()


def pin_python_int_variants():
    """The mpn-style variants (carry-in, one-limb and shorter second
    operands) and the square, against Python's integers."""
    g = W.rng(14)
    for ma, mb in ((1, 0), (1, 1), (2, 1), (3, 1), (7, 3), (32, 32), (33, 1), (129, 64)):
        for cls in W.CLASSES:
            x, _ = W.class_operands(g, cls, 6, ma)
            _, y = W.class_operands(g, cls, 6, max(mb, 1))
            y = np.ascontiguousarray(y[:, :mb])
            cin = g.integers(0, 2, 6).astype(np.uint32) * np.uint32(1 + (ma % 3))   # nonzero counts as 1
            for ci in (None, cin):
                s, c = oracle.add_gen(x, y, ci)
                d, br = oracle.sub_gen(x, y, ci)
                for k in range(6):
                    A = to_int(x[k])
                    B = to_int(y[k]) if mb else 0
                    C = 0 if ci is None else int(ci[k] != 0)
                    assert to_int(s[k]) + int(c[k]) * X ** ma == A + B + C, (ma, mb, cls, k)
                    assert to_int(d[k]) - int(br[k]) * X ** ma == A - B - C, (ma, mb, cls, k)
                    assert int(c[k]) in (0, 1) and int(br[k]) in (0, 1)
    for m in (1, 2, 3, 5, 8, 31, 64, 129):
        for cls in W.CLASSES:
            x, _ = W.class_operands(g, cls, 4, m)
            p = oracle.sqr(x)
            for k in range(x.shape[0]):
                assert to_int(p[k]) == to_int(x[k]) ** 2, (m, cls, k)


def pin_closed_forms_variants():
    for m in (1, 2, 5, 64):
        ones = np.full((1, m), 0xFFFFFFFF, np.uint32)
        zeros = np.zeros((1, m), np.uint32)
        one = np.array([[1]], np.uint32)
        # (X^m - 1) + 0 + carry-in 1 = X^m
        s, c = oracle.add_gen(ones, zeros, np.array([1], np.uint32))
        assert not s.any() and c[0] == 1
        # 0 - 0 - borrow-in 1 = X^m - 1 with borrow 1
        d, br = oracle.sub_gen(zeros, zeros, np.array([1], np.uint32))
        assert (d == 0xFFFFFFFF).all() and br[0] == 1
        # one-limb operand: (X^m - 1) + 1 = X^m (the carry ripples all m limbs)
        s, c = oracle.add_gen(ones, one)
        assert not s.any() and c[0] == 1
        # X^(m-1) - 1 = (X^(m-1) - 1): the borrow ripples to the top limb
        top = zeros.copy()
        top[0, m - 1] = 1
        d, br = oracle.sub_gen(top, one)
        want = np.full(m, 0xFFFFFFFF, np.uint32)
        want[m - 1] = 0
        assert (d[0] == want).all() and br[0] == 0
        # (X^m - 1)^2 = X^2m - 2 X^m + 1: limbs 1, 0.., 0xFFFFFFFE, 0xFFFFFFFF..
        p = oracle.sqr(ones)[0]
        assert p[0] == 1 and not p[1:m].any() and p[m] == 0xFFFFFFFE and (p[m + 1:] == 0xFFFFFFFF).all()


def pin_unsaturated_radix():
    """The radix-2^k product (Sec. 2.1's unsaturated representation) against
    Python's integers, brute force over edge digits, the closed form
    (2^(kn) - 1)^2, and a digit of 2^k or more rejected."""
    g = W.rng(18)
    for bits in (27, 31, 16):
        for n in (1, 2, 3, 5, 8, 31, 64, 129):
            for cls in ("uniform", "max_pair", "zeros", "sparse", "ones"):
                x, y = W.radix_operands(g, cls, 4, n, bits)
                p = oracle.mul_radix(x, y, bits)
                assert p.shape == (4, 2 * n)
                assert int(p.max()) < (1 << bits)
                for k in range(4):
                    assert to_int_radix(p[k], bits) == to_int_radix(x[k], bits) * to_int_radix(y[k], bits), \
                        (bits, n, cls, k)
    bits = 27
    top = (1 << bits) - 1
    edge = np.array([0, 1, 2, 1 << 26, top - 1, top], dtype=np.uint32)
    x = np.repeat(edge, edge.size)[:, None]
    y = np.tile(edge, edge.size)[:, None]
    p = oracle.mul_radix(x, y, bits)
    for k in range(x.shape[0]):
        assert to_int_radix(p[k], bits) == int(x[k, 0]) * int(y[k, 0])
    for n in (1, 4, 40):
        ones = np.full((1, n), top, np.uint32)
        want = from_int_radix(((1 << (bits * n)) - 1) ** 2, 2 * n, bits)
        assert (oracle.mul_radix(ones, ones, bits)[0] == want).all()
        assert want[0] == 1 and want[n] == top - 1 and (want[n + 1:] == top).all()
    bad = np.array([[1 << bits]], np.uint32)
    with pytest.raises(RuntimeError):
        oracle.mul_radix(bad, bad, bits)


PINS = [pin_python_int_addsub, pin_python_int_mul, pin_python_int_mul_columns,
        pin_brute_force_small, pin_closed_forms, pin_invariants,
        pin_column_worked_example, pin_ragged_and_mixed, pin_carry_probability,
        pin_python_int_variants, pin_closed_forms_variants, pin_unsaturated_radix]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


def test_bad_arguments_rejected():
    L = oracle.lib()
    assert L.oracle_add(None, None, None, None, 4, 1) == -1
    assert L.oracle_mul(None, None, None, 4, 1) == -1
    # empty work is fine
    assert L.oracle_add(None, None, None, None, 0, 0) == 0


def test_columns_leave_no_carry_past_2m_limbs():
    """The column form's carry pass ends with no carry for m-limb inputs (the
    product has 2m limbs); the largest operands are the tightest case."""
    ones = np.full((3, 9), 0xFFFFFFFF, dtype=np.uint32)
    oracle.mul_columns(ones, ones)   # raises on a nonzero final carry


def test_threaded_rows_match_single():
    g = W.rng(17)
    x, y = W.class_operands(g, "uniform", 1000, 24)
    s1, c1 = oracle.add(x, y)
    s2, c2 = oracle.add(x, y, threads=4)
    assert (s1 == s2).all() and (c1 == c2).all()
    assert (oracle.mul(x, y) == oracle.mul(x, y, threads=3)).all()
