"""Independent big-integer helpers for the tests: Python's own int (30-bit
digits, its own add/sub/mul) converts limb rows to and from integers.  Shares
nothing with the oracle or the CUDA library."""
import numpy as np

X = 1 << 32


def to_int(limbs) -> int:
    v = 0
    for x in reversed([int(t) for t in np.asarray(limbs).ravel()]):
        v = (v << 32) | x
    return v


def from_int(v: int, m: int) -> np.ndarray:
    out = np.empty(m, dtype=np.uint32)
    for i in range(m):
        out[i] = v & 0xFFFFFFFF
        v >>= 32
    return out


def rows_to_ints(a):
    a = np.asarray(a)
    return [to_int(r) for r in a]


def to_int_radix(digits, bits: int) -> int:
    """Value of little-endian digits in radix 2^bits."""
    v = 0
    for x in reversed([int(t) for t in np.asarray(digits).ravel()]):
        v = (v << bits) | x
    return v


def from_int_radix(v: int, n: int, bits: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    mask = (1 << bits) - 1
    for i in range(n):
        out[i] = v & mask
        v >>= bits
    return out
