"""Seeded synthetic operand generators.

This module is shared by the tests, the bench and the oracle checks.  It draws
random limbs and lays out structured patterns (all-ones limbs, sparse limbs,
long carry/borrow-propagate runs); it performs none of the arithmetic of the
method.  Operands are little-endian arrays of 32-bit limbs, one operand per row
(``uint32[batch][m]``), the saturated-radix layout of Sec. 2.1 with k = 32.

Every generator takes an explicit seed and uses numpy's MT19937 bit generator,
echoing the Mersenne-Twister test-case generation of Sec. 5 (random and
pathological cases).  The five named workloads are:

* ``correctness_mix``   4096 pairs of 1024-bit operands, three value classes
* ``addsub_bandwidth``  2^20 pairs of 4096-bit plus 64 pairs of 2^22-bit operands
                        with long propagate runs
* ``batched_mul``       2^16 pairs at 256/1024/4096/8192 bits
* ``ragged_mixed``      200k mixed add/sub/mul ops, log-uniform 128..16384 bits
* ``shared_operand``    one fixed 2048-bit multiplier and 2^16 2048-bit operands
"""
from __future__ import annotations

import numpy as np

LIMB_MASK = np.uint32(0xFFFFFFFF)
TOP_BIT = np.uint32(0x80000000)

# op codes of the mixed ragged descriptors (mirrors DOT_OP_* in include/dot.h)
OP_ADD, OP_SUB, OP_MUL = 0, 1, 2

# seeds of the five named workloads
SEED_CORRECTNESS_MIX = 1001
SEED_ADDSUB_BANDWIDTH = 1002
SEED_BATCHED_MUL = 1003
SEED_RAGGED_MIXED = 1004
SEED_SHARED_OPERAND = 1005


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.MT19937(seed))


def uniform_limbs(g: np.random.Generator, shape) -> np.ndarray:
    """Independent uniform 32-bit limbs."""
    return g.integers(0, 1 << 32, size=shape, dtype=np.uint32)


def nonzero_limbs(g: np.random.Generator, shape) -> np.ndarray:
    """Uniform limbs on [1, 2^32 - 1]."""
    return g.integers(1, 1 << 32, size=shape, dtype=np.uint32)


def order_pairs(x: np.ndarray, y: np.ndarray):
    """Return (max(x, y), min(x, y)) row by row, comparing from the top limb.

    Only a lexicographic comparison of limb rows; used so that subtraction
    inputs satisfy a >= b where a workload asks for it.
    """
    x = np.ascontiguousarray(x)
    y = np.ascontiguousarray(y)
    if x.shape[1] == 0:
        return x.copy(), y.copy()
    diff = x != y
    # highest differing limb per row (rows that are equal keep x)
    rev = diff[:, ::-1]
    anyd = rev.any(axis=1)
    top = x.shape[1] - 1 - rev.argmax(axis=1)
    rows = np.arange(x.shape[0])
    x_less = anyd & (x[rows, top] < y[rows, top])
    hi = np.where(x_less[:, None], y, x)
    lo = np.where(x_less[:, None], x, y)
    return hi, lo


# --------------------------------------------------------------------------
# small random cases for tests: value classes of Sec. 5
# --------------------------------------------------------------------------
CLASSES = ("uniform", "ones", "zeros", "sparse", "runs", "max_pair")


def class_operands(g: np.random.Generator, cls: str, batch: int, m: int):
    """A pair of operand batches (x, y) of one value class.

    uniform  : uniform limbs
    ones     : x all-ones, y with only limb 0 nonzero (full carry ripple on add)
    zeros    : both zero
    sparse   : each limb nonzero with probability 0.01
    runs     : uniform limbs overlaid with one propagate run per operand
               (x limbs 2^32-1, y limbs 0, preceded by a generating limb pair)
    max_pair : both operands all-ones (largest column sums of a product)
    """
    shape = (batch, m)
    if cls == "uniform":
        return uniform_limbs(g, shape), uniform_limbs(g, shape)
    if cls == "ones":
        x = np.full(shape, LIMB_MASK, dtype=np.uint32)
        y = np.zeros(shape, dtype=np.uint32)
        if m:
            y[:, 0] = nonzero_limbs(g, batch)
        return x, y
    if cls == "zeros":
        return np.zeros(shape, np.uint32), np.zeros(shape, np.uint32)
    if cls == "sparse":
        x = np.where(g.random(shape) < 0.01, nonzero_limbs(g, shape), 0).astype(np.uint32)
        y = np.where(g.random(shape) < 0.01, nonzero_limbs(g, shape), 0).astype(np.uint32)
        return x, y
    if cls == "runs":
        x, y = uniform_limbs(g, shape), uniform_limbs(g, shape)
        if m >= 2:
            start = g.integers(1, m, size=batch)
            length = g.integers(1, m, size=batch)
            idx = np.arange(m)[None, :]
            run = (idx >= start[:, None]) & (idx < (start + length)[:, None])
            x[run] = LIMB_MASK
            y[run] = 0
            rows = np.arange(batch)
            x[rows, start - 1] = TOP_BIT
            y[rows, start - 1] = TOP_BIT
        return x, y
    if cls == "max_pair":
        x = np.full(shape, LIMB_MASK, dtype=np.uint32)
        return x, x.copy()
    raise ValueError(f"unknown class {cls}")


def sub_runs_operands(g: np.random.Generator, batch: int, m: int):
    """Borrow-propagate runs for subtraction: equal limbs preceded by a
    borrow-generating limb pair (x < y at that limb)."""
    x, y = uniform_limbs(g, (batch, m)), uniform_limbs(g, (batch, m))
    if m >= 2:
        start = g.integers(1, m, size=batch)
        length = g.integers(1, m, size=batch)
        idx = np.arange(m)[None, :]
        run = (idx >= start[:, None]) & (idx < (start + length)[:, None])
        y[run] = x[run]
        rows = np.arange(batch)
        x[rows, start - 1] = 0
        y[rows, start - 1] = 1
    return x, y


# --------------------------------------------------------------------------
# the five named workloads
# --------------------------------------------------------------------------
def correctness_mix(seed: int = SEED_CORRECTNESS_MIX, batch: int = 4096, m: int = 32):
    """4096 pairs of 1024-bit operands (32 limbs).

    Each pair falls in one class: 50% uniform limbs; 25% all-ones, where x is
    2^(32m) - 1 and y has only limb 0 nonzero so an addition carry ripples the
    whole length; 25% sparse, each limb nonzero with probability 0.01.
    Subtraction uses (max(x, y), min(x, y)) so a >= b; in the all-ones class it
    uses the borrow dual instead: a has only its top limb nonzero and b only
    limb 0, so the borrow ripples the whole length.  The product uses (x, y).

    Returns dict(x, y, a_sub, b_sub, cls).
    """
    g = rng(seed)
    cls = g.choice(3, size=batch, p=[0.5, 0.25, 0.25])
    x = uniform_limbs(g, (batch, m))
    y = uniform_limbs(g, (batch, m))
    ones = cls == 1
    n1 = int(ones.sum())
    x[ones] = LIMB_MASK
    y[ones] = 0
    y[ones, 0] = nonzero_limbs(g, n1)
    sp = cls == 2
    n2 = int(sp.sum())
    x[sp] = np.where(g.random((n2, m)) < 0.01, nonzero_limbs(g, (n2, m)), 0)
    y[sp] = np.where(g.random((n2, m)) < 0.01, nonzero_limbs(g, (n2, m)), 0)
    a_sub, b_sub = order_pairs(x, y)
    a_sub[ones] = 0
    a_sub[ones, m - 1] = nonzero_limbs(g, n1)
    b_sub[ones] = 0
    b_sub[ones, 0] = nonzero_limbs(g, n1)
    return dict(x=x, y=y, a_sub=a_sub, b_sub=b_sub, cls=cls)


def _overlay_runs_batched(g, x, y, frac, lo_len, hi_len, sub):
    """Overwrite about ``frac`` of all limb positions with one propagate run in
    each of a random subset of rows (run lengths uniform in [lo_len, hi_len])."""
    batch, m = x.shape
    mean_len = 0.5 * (lo_len + hi_len)
    nruns = min(batch, int(round(frac * batch * m / mean_len)))
    rows = g.choice(batch, size=nruns, replace=False)
    length = g.integers(lo_len, hi_len + 1, size=nruns)
    start = 1 + (g.random(nruns) * (m - length)).astype(np.int64)
    idx = np.arange(m)[None, :]
    run = (idx >= start[:, None]) & (idx < (start + length)[:, None])
    xs = x[rows]
    ys = y[rows]
    r = np.arange(nruns)
    if sub:
        ys[run] = xs[run]
        xs[r, start - 1] = 0
        ys[r, start - 1] = 1
    else:
        xs[run] = LIMB_MASK
        ys[run] = 0
        xs[r, start - 1] = TOP_BIT
        ys[r, start - 1] = TOP_BIT
    x[rows] = xs
    y[rows] = ys


def _overlay_runs_long(g, x, y, frac, lo_len, hi_len, sub):
    """Same as above for a few very long rows: runs placed one at a time (rows
    chosen with replacement) until about ``frac`` of the positions are covered."""
    batch, m = x.shape
    target = frac * batch * m
    covered = 0
    while covered < target:
        row = int(g.integers(0, batch))
        length = int(g.integers(lo_len, hi_len + 1))
        start = int(g.integers(1, m - length))
        if sub:
            y[row, start:start + length] = x[row, start:start + length]
            x[row, start - 1] = 0
            y[row, start - 1] = 1
        else:
            x[row, start:start + length] = LIMB_MASK
            y[row, start:start + length] = 0
            x[row, start - 1] = TOP_BIT
            y[row, start - 1] = TOP_BIT
        covered += length


def addsub_bandwidth(seed: int = SEED_ADDSUB_BANDWIDTH, short_batch: int = 1 << 20,
                     short_m: int = 128, long_batch: int = 64, long_m: int = 1 << 17,
                     short_runs=(16, 112), long_runs=(1 << 10, 1 << 16)):
    """Add/sub bandwidth workload.

    Part (i): ``short_batch`` pairs of ``short_m`` limbs (default 2^20 x 4096
    bits).  Part (ii): ``long_batch`` pairs of ``long_m`` limbs (default 64 x
    2^22 bits) whose carry chains cross many thread blocks.  Limbs are uniform;
    then about 10% of limb positions are overwritten by long propagate runs.
    For addition a run is x = 2^32-1, y = 0, preceded by one generating limb
    pair (2^31, 2^31); for subtraction the dual run is x = y, preceded by a
    borrow-generating pair (0, 1).  Row 0 of part (ii) is a full-length ripple:
    (2^n - 1) + 1 for addition and 0 - 1 for subtraction.

    Returns dict with add_short=(x, y), sub_short=(x, y), add_long=(x, y),
    sub_long=(x, y).
    """
    g = rng(seed)
    out = {}
    for name, sub in (("add", False), ("sub", True)):
        xs = uniform_limbs(g, (short_batch, short_m))
        ys = uniform_limbs(g, (short_batch, short_m))
        lo, hi = short_runs
        hi = min(hi, short_m - 2)
        lo = min(lo, hi)
        if short_m >= 4:
            _overlay_runs_batched(g, xs, ys, 0.10, lo, hi, sub)
        xl = uniform_limbs(g, (long_batch, long_m))
        yl = uniform_limbs(g, (long_batch, long_m))
        lo, hi = long_runs
        hi = min(hi, long_m // 2)
        lo = min(lo, hi)
        if long_m >= 8 and long_batch:
            _overlay_runs_long(g, xl, yl, 0.10, lo, hi, sub)
        if long_batch:
            if sub:
                xl[0] = 0
                yl[0] = 0
                yl[0, 0] = 1
            else:
                xl[0] = LIMB_MASK
                yl[0] = 0
                yl[0, 0] = 1
        out[f"{name}_short"] = (xs, ys)
        out[f"{name}_long"] = (xl, yl)
    return out


def batched_mul(m: int, seed: int = SEED_BATCHED_MUL, batch: int = 1 << 16):
    """2^16 pairs of m-limb operands; uniform limbs, and 10% of the pairs have
    both operands all-ones (maximal column sums).  Returns (x, y, maxed)."""
    g = rng(seed + 7919 * m)
    x = uniform_limbs(g, (batch, m))
    y = uniform_limbs(g, (batch, m))
    maxed = g.random(batch) < 0.10
    x[maxed] = LIMB_MASK
    y[maxed] = LIMB_MASK
    return x, y, maxed


BATCHED_MUL_SIZES = (8, 32, 128, 256)


def ragged_sizes(g: np.random.Generator, n: int) -> np.ndarray:
    """Operand limb counts log-uniform over 128..16384 bits:
    m = max(4, round(2^u / 32)) with u ~ U[7, 14]."""
    u = g.uniform(7.0, 14.0, size=n)
    return np.maximum(4, np.rint(np.exp2(u) / 32.0)).astype(np.int64)


def ragged_mixed(seed: int = SEED_RAGGED_MIXED, nops: int = 200_000,
                 frac=(0.3, 0.3, 0.4)):
    """Mixed ragged batch: 30% add, 30% sub, 40% mul, shuffled, sizes from
    ``ragged_sizes``; uniform limbs; subtraction operands ordered so a >= b.

    Packing is CSR-like: operand i occupies a[a_off[i] : a_off[i] + m[i]] and
    b[a_off[i] : ...]; its result occupies r[r_off[i] : r_off[i] + m[i]] for
    add/sub and 2 m[i] limbs for mul; its carry/borrow goes to carry[i].

    Returns dict(op, m, a, b, a_off, r_off, r_len).
    """
    g = rng(seed)
    counts = [int(round(f * nops)) for f in frac]
    counts[2] = nops - counts[0] - counts[1]
    op = np.concatenate([np.full(c, k, dtype=np.uint32) for k, c in enumerate(counts)])
    g.shuffle(op)
    m = ragged_sizes(g, nops)
    a_off = np.zeros(nops + 1, dtype=np.uint64)
    np.cumsum(m, out=a_off[1:])
    total = int(a_off[-1])
    a = uniform_limbs(g, total)
    b = uniform_limbs(g, total)
    # subtraction operands: order each pair so that a >= b (compare from the top)
    for i in np.nonzero(op == OP_SUB)[0]:
        s, e = int(a_off[i]), int(a_off[i + 1])
        av, bv = a[s:e], b[s:e]
        d = np.nonzero(av != bv)[0]
        if d.size and av[d[-1]] < bv[d[-1]]:
            tmp = av.copy()
            a[s:e] = bv
            b[s:e] = tmp
    r_len = np.where(op == OP_MUL, 2 * m, m).astype(np.int64)
    r_off = np.zeros(nops + 1, dtype=np.uint64)
    np.cumsum(r_len, out=r_off[1:])
    return dict(op=op, m=m.astype(np.int64), a=a, b=b, a_off=a_off, r_off=r_off,
                r_len=r_len)


def ragged_uniform(g: np.random.Generator, sizes, cls: str = "uniform"):
    """Pack operands of the given limb counts (one op per entry) CSR-style.
    Returns (a, b, off) with off[i]..off[i+1] the limbs of op i."""
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=off[1:])
    a = np.empty(int(off[-1]), dtype=np.uint32)
    b = np.empty(int(off[-1]), dtype=np.uint32)
    for i, mi in enumerate(sizes):
        x, y = class_operands(g, cls, 1, int(mi))
        a[int(off[i]):int(off[i + 1])] = x[0]
        b[int(off[i]):int(off[i + 1])] = y[0]
    return a, b, off


# unsaturated radix (Sec. 2.1): digits of UNSAT_BITS bits in 32-bit words
UNSAT_BITS = 27
SEED_UNSATURATED = 1006


def radix_operands(g: np.random.Generator, cls: str, batch: int, n: int, bits: int = UNSAT_BITS):
    """A pair of operand batches of n digits in radix 2^bits (each digit
    below 2^bits in a uint32 word), of one class: uniform, max_pair (every
    digit 2^bits - 1), zeros, sparse (digits nonzero with probability 0.01),
    ones (x all maximal digits, y with only digit 0 nonzero)."""
    shape = (batch, n)
    top = 1 << bits
    if cls == "uniform":
        return (g.integers(0, top, size=shape, dtype=np.uint32), g.integers(0, top, size=shape, dtype=np.uint32))
    if cls == "max_pair":
        x = np.full(shape, top - 1, dtype=np.uint32)
        return x, x.copy()
    if cls == "zeros":
        return np.zeros(shape, np.uint32), np.zeros(shape, np.uint32)
    if cls == "sparse":
        x = np.where(g.random(shape) < 0.01, g.integers(1, top, size=shape, dtype=np.uint32), 0).astype(np.uint32)
        y = np.where(g.random(shape) < 0.01, g.integers(1, top, size=shape, dtype=np.uint32), 0).astype(np.uint32)
        return x, y
    if cls == "ones":
        x = np.full(shape, top - 1, dtype=np.uint32)
        y = np.zeros(shape, dtype=np.uint32)
        if n:
            y[:, 0] = g.integers(1, top, size=batch, dtype=np.uint32)
        return x, y
    raise ValueError(f"unknown class {cls}")


def unsaturated_mul(bits_total: int, seed: int = SEED_UNSATURATED, batch: int = 1 << 16,
                    bits: int = UNSAT_BITS):
    """2^16 pairs of ceil(bits_total / bits)-digit operands in radix 2^bits:
    uniform digits, 10% of the pairs both all-maximal digits (largest column
    sums).  Returns (x, y)."""
    n = -(-bits_total // bits)
    g = rng(seed + 7919 * n)
    x, y = radix_operands(g, "uniform", batch, n, bits)
    maxed = g.random(batch) < 0.10
    x[maxed] = (1 << bits) - 1
    y[maxed] = (1 << bits) - 1
    return x, y


def shared_operand(seed: int = SEED_SHARED_OPERAND, batch: int = 1 << 16, m: int = 64):
    """One fixed uniform m-limb multiplier and ``batch`` uniform m-limb
    operands (default 2048-bit).  Returns (fixed[m], b[batch][m])."""
    g = rng(seed)
    return uniform_limbs(g, m), uniform_limbs(g, (batch, m))
