"""CPU oracle for the multi-limb add / sub / mul path -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the bench's CPU-baseline
(and ``--impl reference``) leg may import this package.  The product library
never loads it, and it never loads the product library: the two share no code.

``dot_oracle.c`` holds the arithmetic (Theorem 1 / Theorem 2 definitions, the
row-wise schoolbook, and Theorem 2's column-sum form); this module only compiles it
with gcc and marshals numpy arrays into it.  Every function is pinned by the
``-m "not gpu"`` tests against Python's own big integers, closed forms,
invariants, brute force on <= 64-bit inputs and the m = 5 worked example of
Sec. 3.2 (see tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dot_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_sz = ctypes.c_size_t

_lib = None


def build(force: bool = False) -> str:
    """Compile dot_oracle.c into liboracle.so (portable flags: no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall",
                               "-Wextra", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def bind(path: str):
    """Load a compiled oracle library and declare its signatures."""
    L = ctypes.CDLL(path)
    for name in ("oracle_add", "oracle_sub"):
        f = getattr(L, name)
        f.argtypes = [_u32p, _u32p, _u32p, _u32p, _sz, _sz]
        f.restype = ctypes.c_int
    for name in ("oracle_mul", "oracle_mul_columns"):
        f = getattr(L, name)
        f.argtypes = [_u32p, _u32p, _u32p, _sz, _sz]
        f.restype = ctypes.c_int
    for name in ("oracle_add_ragged", "oracle_sub_ragged"):
        f = getattr(L, name)
        f.argtypes = [_u32p, _u32p, _u32p, _u32p, _u64p, _sz]
        f.restype = ctypes.c_int
    L.oracle_mul_ragged.argtypes = [_u32p, _u32p, _u32p, _u64p, _u64p, _sz]
    L.oracle_mul_ragged.restype = ctypes.c_int
    L.oracle_mixed.argtypes = [_u32p, _u32p, _u64p, _u64p, _u64p, _sz,
                               _u32p, _u32p, _u32p, _u32p]
    L.oracle_mixed.restype = ctypes.c_int
    L.oracle_column_pairs.argtypes = [_sz, _i32p, _i32p, _i32p]
    L.oracle_column_pairs.restype = ctypes.c_int
    for name in ("oracle_add_gen", "oracle_sub_gen"):
        f = getattr(L, name)
        f.argtypes = [_u32p, _sz, _u32p, _sz, _u32p, _u32p, _u32p, _sz]
        f.restype = ctypes.c_int
    L.oracle_sqr.argtypes = [_u32p, _u32p, _sz, _sz]
    L.oracle_sqr.restype = ctypes.c_int
    L.oracle_mul_radix.argtypes = [_u32p, _u32p, _u32p, _sz, _sz, ctypes.c_uint]
    L.oracle_mul_radix.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def _p32(x):
    return x.ctypes.data_as(_u32p)


def _p64(x):
    return x.ctypes.data_as(_u64p)


def _c(x, dtype=np.uint32):
    return np.ascontiguousarray(x, dtype=dtype)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def _batched(a, b):
    a = _c(a)
    b = _c(b)
    if a.shape != b.shape:
        raise ValueError("operand shapes differ")
    if a.ndim == 1:
        a = a[None, :]
        b = b[None, :]
    return a, b


def add(a, b, threads: int = 1):
    """S, carry with S + carry * X^m = A + B, row by row."""
    a, b = _batched(a, b)
    B, m = a.shape
    s = np.empty_like(a)
    c = np.empty(B, dtype=np.uint32)
    _run_rows(lib().oracle_add, a, b, s, c, m, B, threads, out_limbs=m)
    return s, c


def sub(a, b, threads: int = 1):
    """D, borrow with D - borrow * X^m = A - B, row by row."""
    a, b = _batched(a, b)
    B, m = a.shape
    d = np.empty_like(a)
    c = np.empty(B, dtype=np.uint32)
    _run_rows(lib().oracle_sub, a, b, d, c, m, B, threads, out_limbs=m)
    return d, c


def mul(a, b, threads: int = 1):
    """P = A * B as 2m limbs, row by row (row-wise schoolbook)."""
    a, b = _batched(a, b)
    B, m = a.shape
    p = np.empty((B, 2 * m), dtype=np.uint32)
    _run_rows(lib().oracle_mul, a, b, p, None, m, B, threads, out_limbs=2 * m)
    return p


def _gen(fn, what, a, b, cin):
    a = _c(a)
    b = _c(b)
    if a.ndim == 1:
        a, b = a[None, :], b[None, :]
        cin = None if cin is None else np.atleast_1d(cin)
    B, ma = a.shape
    mb = b.shape[1]
    if b.shape[0] != B:
        raise ValueError("operand batches differ")
    s = np.empty_like(a)
    c = np.empty(B, dtype=np.uint32)
    ci = None if cin is None else _c(cin)
    if ci is not None and ci.size != B:
        raise ValueError("carry-in must hold one word per row")
    _check(fn(_p32(a), ma, _p32(b), mb, _p32(ci) if ci is not None else None, _p32(s), _p32(c), B), what)
    return s, c


def add_gen(a, b, cin=None):
    """S, carry with S + carry X^ma = A + B + [cin != 0]; B ([batch][mb], mb <=
    ma) padded with zeros; cin per row or None."""
    return _gen(lib().oracle_add_gen, "oracle_add_gen", a, b, cin)


def sub_gen(a, b, bin=None):
    """D, borrow with D - borrow X^ma = A - B - [bin != 0]; B padded with zeros."""
    return _gen(lib().oracle_sub_gen, "oracle_sub_gen", a, b, bin)


def sqr(a):
    """P = A * A as 2m limbs, row by row."""
    a = _c(a)
    if a.ndim == 1:
        a = a[None, :]
    B, m = a.shape
    p = np.empty((B, 2 * m), dtype=np.uint32)
    _check(lib().oracle_sqr(_p32(a), _p32(p), m, B), "oracle_sqr")
    return p


def mul_radix(a, b, bits: int, threads: int = 1):
    """P = A * B for n-digit operands in radix 2^bits (each digit below 2^bits
    in a 32-bit word), as 2n digits below 2^bits, row by row."""
    a, b = _batched(a, b)
    B, n = a.shape
    p = np.empty((B, 2 * n), dtype=np.uint32)
    L = lib()

    def fn(x, y, z, n_, rows):
        return L.oracle_mul_radix(x, y, z, n_, rows, bits)
    fn.__name__ = "oracle_mul_radix"
    _run_rows(fn, a, b, p, None, n, B, threads, out_limbs=2 * n)
    return p


def mul_columns(a, b):
    """P = A * B (2m limbs) as Theorem 2's column sums S_c = sum_{i+j=c} A_i B_j
    followed by one carry pass."""
    a, b = _batched(a, b)
    B, m = a.shape
    p = np.empty((B, 2 * m), dtype=np.uint32)
    _check(lib().oracle_mul_columns(_p32(a), _p32(b), _p32(p), m, B), "oracle_mul_columns")
    return p


def column_pairs(m: int):
    """The (i, j) pairs of every column c = i + j, column by column, i
    ascending: (i list, j list, pairs per column)."""
    ia = np.empty(m * m, dtype=np.int32)
    jb = np.empty(m * m, dtype=np.int32)
    nc = np.empty(2 * m - 1, dtype=np.int32)
    _check(lib().oracle_column_pairs(m, ia.ctypes.data_as(_i32p), jb.ctypes.data_as(_i32p),
                                     nc.ctypes.data_as(_i32p)), "oracle_column_pairs")
    return ia, jb, nc


def _run_rows(fn, a, b, out, carry, m, B, threads, out_limbs):
    """Call a row-batched oracle function, optionally splitting the rows over
    host threads (ctypes releases the GIL during the call)."""
    def call(lo, hi):
        n = hi - lo
        if n <= 0:
            return 0
        args = [_p32(a[lo:hi]), _p32(b[lo:hi]), _p32(out[lo:hi])]
        if carry is not None:
            args.append(_p32(carry[lo:hi]))
        return fn(*args, m, n)

    # a few long rows still spread over min(threads, B) workers
    workers = min(threads, B)
    if workers <= 1:
        _check(call(0, B), fn.__name__)
        return
    step = (B + workers - 1) // workers
    with ThreadPoolExecutor(max_workers=workers) as ex:
        rcs = list(ex.map(lambda lo: call(lo, min(B, lo + step)), range(0, B, step)))
    for rc in rcs:
        _check(rc, fn.__name__)


def add_ragged(a, b, off):
    a, b, off = _c(a), _c(b), _c(off, np.uint64)
    n = off.size - 1
    s = np.empty_like(a)
    c = np.empty(n, dtype=np.uint32)
    _check(lib().oracle_add_ragged(_p32(a), _p32(b), _p32(s), _p32(c), _p64(off), n),
           "oracle_add_ragged")
    return s, c


def sub_ragged(a, b, off):
    a, b, off = _c(a), _c(b), _c(off, np.uint64)
    n = off.size - 1
    d = np.empty_like(a)
    c = np.empty(n, dtype=np.uint32)
    _check(lib().oracle_sub_ragged(_p32(a), _p32(b), _p32(d), _p32(c), _p64(off), n),
           "oracle_sub_ragged")
    return d, c


def mul_ragged(a, b, off):
    """Products of ragged ops; returns (p, poff) with poff = 2 * off."""
    a, b, off = _c(a), _c(b), _c(off, np.uint64)
    n = off.size - 1
    poff = (2 * off).astype(np.uint64)
    p = np.empty(int(poff[-1]) if n >= 0 else 0, dtype=np.uint32)
    _check(lib().oracle_mul_ragged(_p32(a), _p32(b), _p32(p), _p64(off), _p64(poff), n),
           "oracle_mul_ragged")
    return p, poff


def mixed(op, m, a_off, b_off, r_off, a, b, r_len_total, threads: int = 1):
    """Mixed ragged batch: returns (r, carry).  With threads > 1 the ops are
    split into contiguous ranges, one per host thread; every op writes only
    its own result range and carry slot."""
    op, m = _c(op), _c(m)
    a_off, b_off, r_off = _c(a_off, np.uint64), _c(b_off, np.uint64), _c(r_off, np.uint64)
    a, b = _c(a), _c(b)
    n = op.size
    r = np.zeros(int(r_len_total), dtype=np.uint32)
    # a sentinel, so that a carry slot the oracle failed to write shows
    c = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    L = lib()

    def call(lo, hi):
        return L.oracle_mixed(_p32(op[lo:hi]), _p32(m[lo:hi]), _p64(a_off[lo:hi]), _p64(b_off[lo:hi]),
                              _p64(r_off[lo:hi]), hi - lo, _p32(a), _p32(b), _p32(r), _p32(c[lo:hi]))

    workers = max(1, min(threads, n))
    if workers == 1:
        _check(call(0, n), "oracle_mixed")
        return r, c
    step = (n + workers - 1) // workers
    with ThreadPoolExecutor(max_workers=workers) as ex:
        rcs = list(ex.map(lambda lo: call(lo, min(n, lo + step)), range(0, n, step)))
    for rc in rcs:
        _check(rc, "oracle_mixed")
    return r, c


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1
