"""Thin Python binding of libdot's C ABI (include/dot.h).

Argument marshalling only: every computation runs in the CUDA kernels of
libdot.so.  Operands are torch tensors of dtype int32 or uint32 on the GPU
(the 32 bits of each element are one limb), or numpy uint32 arrays for the
host-buffer variants.  Streams default to torch's current stream.

If libdot.so has not been built, or cannot be loaded, every call raises
DotUnavailable: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdot.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "dot.h")

OK, EINVAL, ECUDA, ENOMEM, ETIMEOUT, EUNSUPPORTED = range(6)
OP_ADD, OP_SUB, OP_MUL = 0, 1, 2
MUL_MAX_LIMBS = 512
UNSAT_BITS = 27
UNSAT_MAX_DIGITS = 512


class DotUnavailable(ImportError):
    """libdot.so is missing or failed to load."""


class DotError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})")


_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_st = ctypes.c_int


class Plan(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("seg_limbs", ctypes.c_int),
                ("lanes_per_op", ctypes.c_int), ("chunks", ctypes.c_int),
                ("tile_limbs", ctypes.c_uint64), ("tiles", ctypes.c_uint64),
                ("m_pad", ctypes.c_uint64)]


class Desc(ctypes.Structure):
    """dot_desc_t: one operation of a mixed ragged batch (32 bytes)."""
    _fields_ = [("op", ctypes.c_uint32), ("m", ctypes.c_uint32), ("a_off", ctypes.c_uint64),
                ("b_off", ctypes.c_uint64), ("r_off", ctypes.c_uint64)]


_SIGS = {
    "dot_abi_version": (ctypes.c_int, []),
    "dot_status_str": (ctypes.c_char_p, [_st]),
    "dot_ctx_create": (_st, [ctypes.POINTER(_vp), ctypes.c_int]),
    "dot_ctx_destroy": (None, [_vp]),
    "dot_ctx_check": (_st, [_vp, _vp]),
    "dot_ctx_set_wait_limit": (_st, [_vp, ctypes.c_uint64]),
    "dot_debug_skip_publish": (_st, [_vp, ctypes.c_int64]),
    "dot_plan_batched": (_st, [ctypes.c_int, _sz, _sz, ctypes.c_int, ctypes.POINTER(Plan)]),
    "dot_add": (_st, [_vp, _vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_sub": (_st, [_vp, _vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_mul": (_st, [_vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_add_ragged": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "dot_sub_ragged": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "dot_mul_ragged": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "dot_mixed_ragged": (_st, [_vp, _vp, _sz, _vp, _vp, _vp, _vp, _vp]),
    "dot_add_host": (_st, [_vp, _vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_sub_host": (_st, [_vp, _vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_mul_host": (_st, [_vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_add_noalloc": (_st, [ctypes.c_int, _vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_mul_shared": (_st, [_vp, _vp, _vp, _vp, _sz, _sz, ctypes.c_int, _vp]),
    "dot_add_nc": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_sub_nc": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_add_1": (_st, [_vp, _vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_sub_1": (_st, [_vp, _vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_add_unequal": (_st, [_vp, _vp, _sz, _vp, _sz, _vp, _vp, _sz, _vp]),
    "dot_sub_unequal": (_st, [_vp, _vp, _sz, _vp, _sz, _vp, _vp, _sz, _vp]),
    "dot_sqr": (_st, [_vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_mul_karatsuba": (_st, [_vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_mul_unsat": (_st, [_vp, _vp, _vp, _vp, _sz, _sz, _vp]),
    "dot_tune_set": (_st, [_vp, ctypes.c_int, _sz, ctypes.c_int]),
    "dot_tune_get": (_st, [_vp, ctypes.c_int, _sz, ctypes.POINTER(ctypes.c_int)]),
    "dot_autotune": (_st, [_vp, ctypes.c_int, _sz, _sz, ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_float)]),
}

_lib = None
_lock = threading.Lock()


def header_functions(path: str = HEADER):
    """Names of the functions include/dot.h declares (DOT_API ...)."""
    text = open(path).read()
    return re.findall(r"DOT_API\s+[\w\s\*]*?\b(dot_\w+)\s*\(", text)


def lib():
    """Load libdot.so once; raise DotUnavailable if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise DotUnavailable(f"{LIB_PATH} is not built (run __graft_entry__.build())")
        try:
            L = ctypes.CDLL(LIB_PATH)
        except OSError as e:  # pragma: no cover
            raise DotUnavailable(f"cannot load {LIB_PATH}: {e}") from e
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_str(status: int) -> str:
    try:
        return lib().dot_status_str(status).decode()
    except DotUnavailable:
        return "status"


def _chk(rc: int, what: str):
    if rc != OK:
        raise DotError(rc, what)


def plan(op: int, m: int, batch: int, vector_ok: bool = True) -> Plan:
    p = Plan()
    _chk(lib().dot_plan_batched(op, m, batch, int(vector_ok), ctypes.byref(p)), "dot_plan_batched")
    return p


# --------------------------------------------------------------- context
class Context:
    """A dot_ctx_t on one CUDA device (owns the library's scratch)."""

    def __init__(self, device: int = 0):
        self.device = device
        h = _vp()
        _chk(lib().dot_ctx_create(ctypes.byref(h), device), "dot_ctx_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib().dot_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def check(self, stream=None) -> int:
        """Synchronise the stream; return the sticky status (and clear it)."""
        return lib().dot_ctx_check(self.handle, _stream(stream))

    def set_wait_limit(self, ns: int):
        _chk(lib().dot_ctx_set_wait_limit(self.handle, int(ns)), "dot_ctx_set_wait_limit")

    def debug_skip_publish(self, tile: int):
        _chk(lib().dot_debug_skip_publish(self.handle, int(tile)), "dot_debug_skip_publish")

    def tune_set(self, op: int, m: int, value: int):
        _chk(lib().dot_tune_set(self.handle, op, m, value), "dot_tune_set")

    def tune_get(self, op: int, m: int) -> int:
        v = ctypes.c_int()
        _chk(lib().dot_tune_get(self.handle, op, m, ctypes.byref(v)), "dot_tune_get")
        return v.value

    def autotune(self, op: int, m: int, batch: int):
        """Time the candidate shapes for (op, m) and keep the fastest in this
        context; returns (knob, ms per call)."""
        best, ms = ctypes.c_int(), ctypes.c_float()
        _chk(lib().dot_autotune(self.handle, op, m, batch, ctypes.byref(best), ctypes.byref(ms)),
             "dot_autotune")
        return best.value, ms.value


_default_ctx = {}


def default_context(device: int | None = None) -> Context:
    import torch
    if device is None:
        device = torch.cuda.current_device()
    c = _default_ctx.get(device)
    if c is None:
        c = Context(device)
        _default_ctx[device] = c
    return c


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


def _ptr(t):
    return _vp(t.data_ptr()) if t is not None else _vp(0)


def _limb_tensor(t, name):
    import torch
    if t.dtype not in (torch.int32, torch.uint32):
        raise TypeError(f"{name}: limbs are 32-bit (int32 or uint32), got {t.dtype}")
    if not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    return t


# ----------------------------------------------------------- operations
def _addsub(fn, what, a, b, out, carry, ctx, stream):
    _limb_tensor(a, "a"), _limb_tensor(b, "b"), _limb_tensor(out, "out"), _limb_tensor(carry, "carry")
    if a.dim() != 2 or a.shape != b.shape or out.shape != a.shape:
        raise ValueError(f"{what}: a, b, out must be [batch, m] of one shape")
    batch, m = a.shape
    if carry.numel() != batch:
        raise ValueError(f"{what}: carry must hold batch entries")
    ctx = ctx or default_context(a.device.index)
    _chk(fn(ctx.handle, _ptr(a), _ptr(b), _ptr(out), _ptr(carry), m, batch, _stream(stream)), what)
    return out, carry


def add(a, b, out=None, carry=None, ctx=None, stream=None):
    """(s, carry) with s + carry X^m = a + b, row by row (Alg. 1)."""
    import torch
    out = torch.empty_like(a) if out is None else out
    carry = torch.empty(a.shape[0], dtype=a.dtype, device=a.device) if carry is None else carry
    return _addsub(lib().dot_add, "dot_add", a, b, out, carry, ctx, stream)


def sub(a, b, out=None, borrow=None, ctx=None, stream=None):
    """(d, borrow) with d - borrow X^m = a - b, row by row."""
    import torch
    out = torch.empty_like(a) if out is None else out
    borrow = torch.empty(a.shape[0], dtype=a.dtype, device=a.device) if borrow is None else borrow
    return _addsub(lib().dot_sub, "dot_sub", a, b, out, borrow, ctx, stream)


def mul(a, b, out=None, ctx=None, stream=None):
    """p = a * b as 2m limbs, row by row (Alg. 2)."""
    import torch
    _limb_tensor(a, "a"), _limb_tensor(b, "b")
    if a.dim() != 2 or a.shape != b.shape:
        raise ValueError("dot_mul: a, b must be [batch, m] of one shape")
    batch, m = a.shape
    if out is None:
        out = torch.empty((batch, 2 * m), dtype=a.dtype, device=a.device)
    _limb_tensor(out, "out")
    if tuple(out.shape) != (batch, 2 * m):
        raise ValueError("dot_mul: out must be [batch, 2m]")
    ctx = ctx or default_context(a.device.index)
    _chk(lib().dot_mul(ctx.handle, _ptr(a), _ptr(b), _ptr(out), m, batch, _stream(stream)), "dot_mul")
    return out


def _carry_like(a, carry):
    import torch
    return torch.empty(a.shape[0], dtype=a.dtype, device=a.device) if carry is None else carry


def add_nc(a, b, carry_in, out=None, carry=None, ctx=None, stream=None, sub=False):
    """(s, carry) with s + carry X^m = a + b + [carry_in != 0], row by row
    (with sub=True: d - borrow X^m = a - b - [borrow_in != 0])."""
    import torch
    out = torch.empty_like(a) if out is None else out
    carry = _carry_like(a, carry)
    for t, n in ((a, "a"), (b, "b"), (carry_in, "carry_in"), (out, "out"), (carry, "carry")):
        _limb_tensor(t, n)
    what = "dot_sub_nc" if sub else "dot_add_nc"
    if a.dim() != 2 or a.shape != b.shape or out.shape != a.shape or carry_in.numel() != a.shape[0] \
            or carry.numel() != a.shape[0]:
        raise ValueError(f"{what}: a, b, out [batch, m]; carry_in, carry [batch]")
    batch, m = a.shape
    ctx = ctx or default_context(a.device.index)
    fn = lib().dot_sub_nc if sub else lib().dot_add_nc
    _chk(fn(ctx.handle, _ptr(a), _ptr(b), _ptr(carry_in), _ptr(out), _ptr(carry), m, batch, _stream(stream)),
         what)
    return out, carry


def sub_nc(a, b, borrow_in, out=None, borrow=None, ctx=None, stream=None):
    return add_nc(a, b, borrow_in, out, borrow, ctx, stream, sub=True)


def add_1(a, b, out=None, carry=None, ctx=None, stream=None, sub=False):
    """(s, carry) with s + carry X^m = a + b for a one-limb b[k] per row."""
    import torch
    out = torch.empty_like(a) if out is None else out
    carry = _carry_like(a, carry)
    for t, n in ((a, "a"), (b, "b"), (out, "out"), (carry, "carry")):
        _limb_tensor(t, n)
    what = "dot_sub_1" if sub else "dot_add_1"
    if a.dim() != 2 or out.shape != a.shape or b.numel() != a.shape[0] or carry.numel() != a.shape[0]:
        raise ValueError(f"{what}: a, out [batch, m]; b, carry [batch]")
    batch, m = a.shape
    ctx = ctx or default_context(a.device.index)
    fn = lib().dot_sub_1 if sub else lib().dot_add_1
    _chk(fn(ctx.handle, _ptr(a), _ptr(b), _ptr(out), _ptr(carry), m, batch, _stream(stream)), what)
    return out, carry


def sub_1(a, b, out=None, borrow=None, ctx=None, stream=None):
    return add_1(a, b, out, borrow, ctx, stream, sub=True)


def add_unequal(a, b, out=None, carry=None, ctx=None, stream=None, sub=False):
    """(s, carry) with s + carry X^ma = a + b for a: [batch, ma], b: [batch, mb], mb <= ma."""
    import torch
    out = torch.empty_like(a) if out is None else out
    carry = _carry_like(a, carry)
    for t, n in ((a, "a"), (b, "b"), (out, "out"), (carry, "carry")):
        _limb_tensor(t, n)
    what = "dot_sub_unequal" if sub else "dot_add_unequal"
    if a.dim() != 2 or b.dim() != 2 or b.shape[0] != a.shape[0] or out.shape != a.shape \
            or carry.numel() != a.shape[0]:
        raise ValueError(f"{what}: a, out [batch, ma]; b [batch, mb]; carry [batch]")
    batch, ma = a.shape
    mb = b.shape[1]
    ctx = ctx or default_context(a.device.index)
    fn = lib().dot_sub_unequal if sub else lib().dot_add_unequal
    _chk(fn(ctx.handle, _ptr(a), ma, _ptr(b), mb, _ptr(out), _ptr(carry), batch, _stream(stream)), what)
    return out, carry


def sub_unequal(a, b, out=None, borrow=None, ctx=None, stream=None):
    return add_unequal(a, b, out, borrow, ctx, stream, sub=True)


def mul_karatsuba(a, b, out=None, ctx=None, stream=None):
    """p = a * b as 2m limbs for any m: Karatsuba levels above the base case."""
    import torch
    _limb_tensor(a, "a"), _limb_tensor(b, "b")
    if a.dim() != 2 or a.shape != b.shape:
        raise ValueError("dot_mul_karatsuba: a, b must be [batch, m] of one shape")
    batch, m = a.shape
    if out is None:
        out = torch.empty((batch, 2 * m), dtype=a.dtype, device=a.device)
    _limb_tensor(out, "out")
    if tuple(out.shape) != (batch, 2 * m):
        raise ValueError("dot_mul_karatsuba: out must be [batch, 2m]")
    ctx = ctx or default_context(a.device.index)
    _chk(lib().dot_mul_karatsuba(ctx.handle, _ptr(a), _ptr(b), _ptr(out), m, batch, _stream(stream)),
         "dot_mul_karatsuba")
    return out


def mul_unsat(a, b, out=None, ctx=None, stream=None):
    """p = a * b for n-digit operands in radix 2^27 (each digit below 2^27 in
    a 32-bit word), as 2n digits below 2^27, row by row."""
    import torch
    _limb_tensor(a, "a"), _limb_tensor(b, "b")
    if a.dim() != 2 or a.shape != b.shape:
        raise ValueError("dot_mul_unsat: a, b must be [batch, n] of one shape")
    batch, n = a.shape
    if out is None:
        out = torch.empty((batch, 2 * n), dtype=a.dtype, device=a.device)
    _limb_tensor(out, "out")
    if tuple(out.shape) != (batch, 2 * n):
        raise ValueError("dot_mul_unsat: out must be [batch, 2n]")
    ctx = ctx or default_context(a.device.index)
    _chk(lib().dot_mul_unsat(ctx.handle, _ptr(a), _ptr(b), _ptr(out), n, batch, _stream(stream)), "dot_mul_unsat")
    return out


def sqr(a, out=None, ctx=None, stream=None):
    """p = a^2 as 2m limbs, row by row (half the partial products of mul)."""
    import torch
    _limb_tensor(a, "a")
    if a.dim() != 2:
        raise ValueError("dot_sqr: a must be [batch, m]")
    batch, m = a.shape
    if out is None:
        out = torch.empty((batch, 2 * m), dtype=a.dtype, device=a.device)
    _limb_tensor(out, "out")
    if tuple(out.shape) != (batch, 2 * m):
        raise ValueError("dot_sqr: out must be [batch, 2m]")
    ctx = ctx or default_context(a.device.index)
    _chk(lib().dot_sqr(ctx.handle, _ptr(a), _ptr(out), m, batch, _stream(stream)), "dot_sqr")
    return out


def mul_shared(fixed, b, out=None, tensor_cores=True, ctx=None, stream=None):
    """p[k] = fixed * b[k] (2m limbs) for one fixed m-limb operand; on the
    tensor cores (m <= 64) or on the INT32 column-sum path."""
    import torch
    _limb_tensor(fixed, "fixed"), _limb_tensor(b, "b")
    if b.dim() != 2 or fixed.numel() != b.shape[1]:
        raise ValueError("dot_mul_shared: fixed is [m], b is [batch, m]")
    batch, m = b.shape
    if out is None:
        out = torch.empty((batch, 2 * m), dtype=b.dtype, device=b.device)
    _limb_tensor(out, "out")
    ctx = ctx or default_context(b.device.index)
    _chk(lib().dot_mul_shared(ctx.handle, _ptr(fixed), _ptr(b), _ptr(out), m, batch, int(bool(tensor_cores)),
                              _stream(stream)), "dot_mul_shared")
    return out


def _off_tensor(off, name):
    import torch
    if off.dtype not in (torch.int64, torch.uint64) or not off.is_cuda or not off.is_contiguous():
        raise TypeError(f"{name}: offsets are a contiguous int64 CUDA tensor")
    return off


def add_ragged(a, b, off, out=None, carry=None, ctx=None, stream=None, sub=False):
    import torch
    _limb_tensor(a, "a"), _limb_tensor(b, "b"), _off_tensor(off, "off")
    n = off.numel() - 1
    out = torch.empty_like(a) if out is None else out
    carry = torch.empty(max(n, 0), dtype=a.dtype, device=a.device) if carry is None else carry
    ctx = ctx or default_context(a.device.index)
    fn = lib().dot_sub_ragged if sub else lib().dot_add_ragged
    _chk(fn(ctx.handle, _ptr(a), _ptr(b), _ptr(out), _ptr(carry), _ptr(off), max(n, 0),
            _stream(stream)), "dot_sub_ragged" if sub else "dot_add_ragged")
    return out, carry


def sub_ragged(a, b, off, out=None, borrow=None, ctx=None, stream=None):
    return add_ragged(a, b, off, out, borrow, ctx, stream, sub=True)


def mul_ragged(a, b, off, poff, out, ctx=None, stream=None):
    _limb_tensor(a, "a"), _limb_tensor(b, "b"), _limb_tensor(out, "out")
    _off_tensor(off, "off"), _off_tensor(poff, "poff")
    n = off.numel() - 1
    ctx = ctx or default_context(a.device.index)
    _chk(lib().dot_mul_ragged(ctx.handle, _ptr(a), _ptr(b), _ptr(out), _ptr(off), _ptr(poff),
                              max(n, 0), _stream(stream)), "dot_mul_ragged")
    return out


def mixed_ragged(desc, a, b, r, carry, ctx=None, stream=None):
    """desc: uint8 CUDA tensor of nops * 32 bytes (dot_desc_t records)."""
    _limb_tensor(a, "a"), _limb_tensor(b, "b"), _limb_tensor(r, "r"), _limb_tensor(carry, "carry")
    nops = desc.numel() // 32
    ctx = ctx or default_context(a.device.index)
    _chk(lib().dot_mixed_ragged(ctx.handle, _ptr(desc), nops, _ptr(a), _ptr(b), _ptr(r), _ptr(carry),
                                _stream(stream)), "dot_mixed_ragged")
    return r, carry


def add_noalloc(a, b, out=None, carry=None, stream=None):
    """dot_add_noalloc: the addition of add() through the entry point that
    performs no device allocation (its scratch is a fixed array inside the
    library; no context).  Calls must not overlap on the GPU."""
    import torch
    out = torch.empty_like(a) if out is None else out
    carry = torch.empty(a.shape[0], dtype=a.dtype, device=a.device) if carry is None else carry
    _limb_tensor(a, "a"), _limb_tensor(b, "b"), _limb_tensor(out, "out"), _limb_tensor(carry, "carry")
    if a.dim() != 2 or a.shape != b.shape or out.shape != a.shape or carry.numel() != a.shape[0]:
        raise ValueError("dot_add_noalloc: a, b, out must be [batch, m]; carry [batch]")
    batch, m = a.shape
    _chk(lib().dot_add_noalloc(a.device.index, _ptr(a), _ptr(b), _ptr(out), _ptr(carry), m, batch,
                               _stream(stream)), "dot_add_noalloc")
    return out, carry


# ------------------------------------------------- host-buffer variants
def _np_ptr(x):
    return _vp(x.ctypes.data) if x is not None else _vp(0)


def host_op(op: int, a, b, out, carry=None, ctx=None, stream=None):
    """Run add/sub/mul on host (numpy uint32) buffers through the library's
    copy-in / compute / copy-out pipeline.  Asynchronous on `stream`: the
    outputs are valid after ctx.check(stream)."""
    batch, m = a.shape
    ctx = ctx or default_context()
    L = lib()
    if op == OP_MUL:
        rc = L.dot_mul_host(ctx.handle, _np_ptr(a), _np_ptr(b), _np_ptr(out), m, batch, _stream(stream))
    else:
        fn = L.dot_add_host if op == OP_ADD else L.dot_sub_host
        rc = fn(ctx.handle, _np_ptr(a), _np_ptr(b), _np_ptr(out), _np_ptr(carry), m, batch, _stream(stream))
    _chk(rc, "dot_*_host")
