"""Binding of libdotprobe (include/dot_probe.h): the microbenchmarks that give
the integer-pipe peaks the multiply kernels are reported against, and the
tensor-pipe rate of each product shape the fixed-operand multiply issues.

``measure()`` runs each probe over the whole GPU (every SM at its full
resident occupancy) for a few tens of milliseconds per launch and returns
rates per second.  The probes compute nothing a caller uses.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdotprobe.so")

MUL_PAIR, COLSUM_R8, MADWIDE_R8, MUL_LO, EMPTY, MMA_N128_TMEM, MMA_N128_SMEM, MMA_N256_TMEM = range(8)
THREADS = 256

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        L.dotp_run.argtypes = [ctypes.c_int] * 5 + [ctypes.POINTER(ctypes.c_float),
                                                     ctypes.POINTER(ctypes.c_double)]
        L.dotp_run.restype = ctypes.c_int
        L.dotp_occupancy.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]
        L.dotp_occupancy.restype = ctypes.c_int
        _lib = L
    return _lib


def occupancy(kind: int, threads: int = THREADS):
    sms, per = ctypes.c_int(), ctypes.c_int()
    rc = lib().dotp_occupancy(kind, threads, ctypes.byref(sms), ctypes.byref(per))
    if rc != 0:
        raise RuntimeError(f"dotp_occupancy failed ({rc})")
    return sms.value, per.value


def run(kind: int, blocks: int, iters: int, reps: int = 5, threads: int = THREADS):
    """(mean ms per launch, units per launch)."""
    ms, units = ctypes.c_float(), ctypes.c_double()
    rc = lib().dotp_run(kind, blocks, threads, iters, reps, ctypes.byref(ms), ctypes.byref(units))
    if rc != 0:
        raise RuntimeError(f"dotp_run({kind}) failed ({rc})")
    return ms.value, units.value


def measure(target_ms: float = 25.0, reps: int = 5):
    """Rates of every probe on the current device, each at full occupancy:
    {name: {"per_s": units per second, "ms": ..., "grid": ..., "unit": ...}}."""
    names = {MUL_PAIR: ("mul_pair", "limb product (mul.lo + mul.hi pair)"),
             COLSUM_R8: ("colsum_r8", "limb product (multiply pair + 3-word add chain)"),
             MADWIDE_R8: ("madwide_r8", "digit product (mad.wide.u32 into 64 bits)"),
             MUL_LO: ("mul_lo", "32-bit multiply (mul.lo.u32)"),
             MMA_N128_TMEM: ("mma_n128_tmem", "flop (tcgen05.mma M=128 N=128 K=16, A in tensor memory)"),
             MMA_N128_SMEM: ("mma_n128_smem", "flop (tcgen05.mma M=128 N=128 K=16, A in shared memory)"),
             MMA_N256_TMEM: ("mma_n256_tmem", "flop (tcgen05.mma M=128 N=256 K=16, A in tensor memory)")}
    out = {}
    for kind, (name, unit) in names.items():
        sms, per = occupancy(kind)
        blocks = sms * per
        # size the loop from a short first run so that a launch lasts ~target_ms
        iters = 256
        ms, units = run(kind, blocks, iters, reps=1)
        if ms > 0:
            iters = max(256, int(iters * target_ms / ms))
        ms, units = run(kind, blocks, iters, reps=reps)
        out[name] = {"per_s": units / (ms * 1e-3), "ms": round(ms, 4), "grid": f"{blocks} x {THREADS}",
                     "blocks_per_sm": per, "unit": unit}
    sms, _ = occupancy(EMPTY)
    ms, _ = run(EMPTY, sms, 1, reps=200)
    out["launch_floor"] = {"us": round(ms * 1e3, 3), "grid": f"{sms} x {THREADS}",
                           "unit": "back-to-back empty launches on one stream"}
    return out
