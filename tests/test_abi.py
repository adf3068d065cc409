"""The C-ABI library builds, loads and exports every symbol include/dot.h
declares; host-side logic (argument checks, launch plans) needs no GPU."""
import ctypes

import pytest

from paper_2604_21566_gb300 import build as B
from paper_2604_21566_gb300 import dot


@pytest.fixture(scope="module")
def L():
    B.build()
    return dot.lib()


def test_exports_every_declared_symbol(L):
    names = dot.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(names) <= set(dot._SIGS), set(names) - set(dot._SIGS)


def test_status_strings_and_version(L):
    assert L.dot_abi_version() == 1
    for code in range(6):
        assert L.dot_status_str(code)
    assert L.dot_status_str(99) == b"unknown status"


def test_null_context_rejected_without_gpu(L):
    v = ctypes.c_void_p
    assert L.dot_add(None, v(0), v(0), v(0), v(0), 4, 4, None) == dot.EINVAL
    assert L.dot_mul(None, v(0), v(0), v(0), 4, 4, None) == dot.EINVAL
    assert L.dot_ctx_create(None, 0) == dot.EINVAL
    assert L.dot_ctx_set_wait_limit(None, 5) == dot.EINVAL
    L.dot_ctx_destroy(None)


def test_plans():
    # whole ops inside a warp
    p = dot.plan(dot.OP_ADD, 128, 1 << 20)
    assert (p.kernel, p.seg_limbs, p.lanes_per_op, p.chunks) == (1, 4, 32, 1)
    p = dot.plan(dot.OP_ADD, 32, 4096)
    assert (p.kernel, p.lanes_per_op, p.chunks) == (1, 8, 1)
    p = dot.plan(dot.OP_SUB, 512, 10)
    assert (p.kernel, p.lanes_per_op, p.chunks) == (1, 32, 4)
    p = dot.plan(dot.OP_ADD, 7, 10, vector_ok=False)
    assert (p.kernel, p.seg_limbs, p.lanes_per_op) == (1, 1, 7)
    # long operands: tiles chained by look-back
    p = dot.plan(dot.OP_ADD, 1 << 17, 64)
    assert p.kernel == 2 and p.tile_limbs == 4096 and p.tiles == 32
    p = dot.plan(dot.OP_ADD, 513, 3)
    assert p.kernel == 2 and p.tiles == 1
    # multiply: up to 16 limbs one product per thread
    for m in (1, 5, 8, 16):
        p = dot.plan(dot.OP_MUL, m, 1000)
        assert (p.kernel, p.lanes_per_op) == (4, 1), m
    # above: two column blocks per lane, R columns each
    for m, R, T in ((17, 8, 3), (32, 8, 4), (128, 8, 16), (256, 8, 32), (512, 16, 32), (100, 8, 13),
                    (96, 12, 8), (150, 16, 10), (192, 12, 16), (300, 12, 25), (384, 12, 32), (385, 16, 25)):
        p = dot.plan(dot.OP_MUL, m, 1)
        assert (p.kernel, p.seg_limbs, p.lanes_per_op) == (3, R, T), m
        assert p.m_pad == R * T


def test_mul_columns_fill_the_warp():
    """Above 16 limbs the default columns per lane R is the one of 8, 12, 16
    that leaves the fewest lane-steps idle: a warp holds floor(32 / T) ops of
    T = ceil(m / R) lanes, each lane summing m' + R rows of R columns."""
    from fractions import Fraction

    def useful(m, R):
        T = -(-m // R)
        return Fraction((32 // T) * m * m, 32 * (T * R + R) * R)

    for m in range(17, 513):
        cands = [R for R in (8, 12, 16) if m <= 32 * R]
        best = max(useful(m, R) for R in cands)
        want = min(R for R in cands if useful(m, R) == best)
        assert dot.plan(dot.OP_MUL, m, 1).seg_limbs == want, m
    with pytest.raises(dot.DotError):
        dot.plan(dot.OP_MUL, 513, 1)
    with pytest.raises(dot.DotError):
        dot.plan(7, 4, 1)
    assert dot.plan(dot.OP_ADD, 4, 0).kernel == 0
    # 17..32 limbs: one product per thread only for batches of at least 2^14
    assert (dot.plan(dot.OP_MUL, 32, 1 << 16).kernel, dot.plan(dot.OP_MUL, 32, 1 << 16).seg_limbs) == (4, 32)
    assert dot.plan(dot.OP_MUL, 17, 1 << 14).kernel == 4
    assert dot.plan(dot.OP_MUL, 32, 4096).kernel == 3
    assert dot.plan(dot.OP_MUL, 33, 1 << 16).kernel == 3


def test_probe_library_exports():
    """libdotprobe (the bench's integer-pipe microbenchmarks) builds and
    exports what include/dot_probe.h declares."""
    import os
    import re
    B.build()
    lib = ctypes.CDLL(os.path.join(os.path.dirname(B.__file__), "libdotprobe.so"))
    hdr = open(os.path.join(B.INCLUDE, "dot_probe.h")).read()
    names = re.findall(r"DOTP_API\s+[\w\s\*]*?\b(dotp_\w+)\s*\(", hdr)
    assert set(names) == {"dotp_run", "dotp_occupancy"}
    for n in names:
        assert hasattr(lib, n), n
    # argument checks need no GPU
    ms, units = ctypes.c_float(), ctypes.c_double()
    assert lib.dotp_run(99, 1, 32, 1, 1, ctypes.byref(ms), ctypes.byref(units)) == 1000
