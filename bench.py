#!/usr/bin/env python3
"""Benchmark of the carry-decoupled add/sub hot path on the GB300.

Workload (one "step"): the add/sub bandwidth set -- 2^20 pairs of 4096-bit
operands plus 64 pairs of 2^22-bit operands (carries crossing thread blocks
through decoupled look-back), uniform limbs with ~10% long propagate runs --
run through dot_add and dot_sub (4 library calls).  Inputs already sit in HBM
when the timed region starts; they are far larger than L2 (1.7 GB per op type),
so no L2 flush is needed between steps.

Prints one JSON line (rank 0).  Metric: bignum operations per second
(Gop/s, every result bit-exact).  ``e2e`` times the same step through the
host-buffer C-ABI entry points (copies in and out inside the timed region).
``--impl reference`` times the CPU oracle on the machine's host cores on a
bounded sample of the same workload instead.

Multi-GPU: the ops are independent, so N ranks run N replicas of the step
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gop/s bit-exact add/sub/mul per operand size; % HBM or int-pipe roofline"
WORKLOAD = "add/sub bandwidth: 2^20 x 4096-bit + 64 x 2^22-bit operand pairs, add and sub"
PROFILE = os.path.join(ROOT, "profiles", "addsub_warp_kernel_4096bit.md")
CSRC = os.path.join(ROOT, "paper_2604_21566_gb300", "csrc")
KERNEL_HEADERS = ("dot_internal.cuh", "dot_addsub.cuh", "dot_plan.h")


def kernel_source_hash() -> str:
    """Hash of the dominant kernel's code: its headers plus the text of
    addsub_warp_kernel and its launcher in dot_addsub.cu."""
    h = hashlib.sha256()
    for f in KERNEL_HEADERS:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    src = open(os.path.join(CSRC, "dot_addsub.cu")).read()
    lo = src.index("// ======================================================= warp kernel (1)")
    hi = src.index("// ================================================= tiled kernel (2)")
    h.update(src[lo:hi].encode())
    lo = src.index("template <bool SUB, int SEG>\nstatic cudaError_t launch_warp")
    hi = src.index("template <bool SUB, int SEG>\nstatic dot_status_t launch_tile")
    h.update(src[lo:hi].encode())
    return h.hexdigest()[:16]


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (replicas report the whole job's throughput
    against it); a barrier follows so no rank races ahead."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job rate in units per second x 1e-9: every rank processes the
    same units (weak scaling), timed by the slowest rank."""
    return world * units_per_rank / (ms * 1e-3) / 1e9


def algorithmic_bytes(m: int, batch: int) -> int:
    """Operands read once (8m bytes), result written once (4m) plus the
    4-byte carry, per op."""
    return batch * (12 * m + 4)


def read_traffic():
    """dram bytes per launch of the dominant kernel from the committed ncu
    summary, or None if missing or taken on different kernel sources."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    vals = {}
    for ln in text.splitlines():
        if ":" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return int(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the GPU works."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- GPU arm
def gpu_arm(args, rank, world, local):
    import torch
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    data = W.addsub_bandwidth()
    ctx = dot.Context(local)

    def to_dev(x):
        return torch.from_numpy(x.view(np.int32)).to(dev)

    parts = []   # (op, x, y, s, c) on the device
    for name in ("add_short", "add_long", "sub_short", "sub_long"):
        x, y = data[name]
        a, b = to_dev(x), to_dev(y)
        s = torch.empty_like(a)
        c = torch.empty(a.shape[0], dtype=torch.int32, device=dev)
        parts.append((name, a, b, s, c))
    stream = torch.cuda.current_stream(dev)
    L = dot.lib()

    def call(name, a, b, s, c):
        fn = L.dot_add if name.startswith("add") else L.dot_sub
        rc = fn(ctx.handle, dot._ptr(a), dot._ptr(b), dot._ptr(s), dot._ptr(c),
                a.shape[1], a.shape[0], dot._stream(stream))
        if rc != dot.OK:
            raise dot.DotError(rc, name)

    ev = {p[0]: [] for p in parts}

    def step(record=False):
        for name, a, b, s, c in parts:
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call(name, a, b, s, c)
                e1.record(stream)
                ev[name].append((e0, e1))
            else:
                call(name, a, b, s, c)

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if ctx.check(stream) != dot.OK:
        raise RuntimeError("device status after warm-up")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1)
    st = ctx.check(stream)
    if st != dot.OK:
        raise RuntimeError(f"device status {st} after the timed region")
    ms = max_over_ranks(ms, world, dev)

    per_launch = {k: sum(e0.elapsed_time(e1) for e0, e1 in v) / len(v) for k, v in ev.items()}
    ops_step = sum(p[1].shape[0] for p in parts)

    # parity of the last step's results on sampled rows (outside the timed region)
    import oracle
    exact = True
    g = np.random.default_rng(7)
    for name, a, b, s, c in parts:
        x, y = data[name]
        rows = np.unique(np.concatenate([[0, x.shape[0] - 1], g.integers(0, x.shape[0], 256)]))
        ws, wc = (oracle.add if name.startswith("add") else oracle.sub)(x[rows], y[rows])
        hs = s[torch.from_numpy(rows).to(dev)].cpu().numpy().view(np.uint32)
        hc = c.cpu().numpy().view(np.uint32)[rows]
        exact &= bool(np.array_equal(hs, ws) and np.array_equal(hc, wc))

    # end to end through the host-buffer entry points, pinned host memory
    pinned = []
    for name in ("add_short", "add_long", "sub_short", "sub_long"):
        x, y = data[name]
        xs = torch.from_numpy(x.view(np.int32)).pin_memory()
        ys = torch.from_numpy(y.view(np.int32)).pin_memory()
        so = torch.empty_like(xs).pin_memory()
        co = torch.empty(x.shape[0], dtype=torch.int32).pin_memory()
        pinned.append((name, xs, ys, so, co))

    def e2e_step():
        for name, xs, ys, so, co in pinned:
            fn = L.dot_add_host if name.startswith("add") else L.dot_sub_host
            rc = fn(ctx.handle, dot._vp(xs.data_ptr()), dot._vp(ys.data_ptr()),
                    dot._vp(so.data_ptr()), dot._vp(co.data_ptr()), xs.shape[1], xs.shape[0],
                    dot._stream(stream))
            if rc != dot.OK:
                raise dot.DotError(rc, name)

    e2e_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    if ctx.check(stream) != dot.OK:
        raise RuntimeError("device status after the end-to-end pass")
    h2d = sum(p[1].numel() * 4 * 2 for p in pinned)
    d2h = sum(p[1].numel() * 4 + p[1].shape[0] * 4 for p in pinned)
    for name, xs, ys, so, co in pinned[:1]:
        x, y = data[name]
        ws, wc = oracle.add(x[:512], y[:512])
        exact &= bool(np.array_equal(so.numpy().view(np.uint32)[:512], ws))
    clocks = sampler.stop()
    e2e_ms = max_over_ranks(e2e_ms, world, dev)

    if rank == 0:
        hbm, src = peaks()
        dom = "add_short"
        dom_ms = 0.5 * (per_launch["add_short"] + per_launch["sub_short"])
        x, _ = data[dom]
        alg = algorithmic_bytes(x.shape[1], x.shape[0])
        achieved = alg / (dom_ms * 1e-3) / 1e9
        parts_out = {}
        for name in per_launch:
            x, _ = data[name]
            parts_out[name] = {
                "m_limbs": int(x.shape[1]), "ops": int(x.shape[0]),
                "ms": round(per_launch[name], 4),
                "gop_s": round(x.shape[0] / (per_launch[name] * 1e-3) / 1e9, 4),
                "GB_s": round(algorithmic_bytes(x.shape[1], x.shape[0]) / (per_launch[name] * 1e-3) / 1e9, 1),
            }
        cpu = cpu_baseline(data, args.cpu_seconds) if not args.no_cpu else None
        ms_step = ms / args.steps
        value = job_throughput(ops_step, world, ms_step)
        out = {
            "metric": METRIC, "value": round(value, 4), "unit": "Gop/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded MT19937, uniform limbs + 10% propagate runs)",
            "config": {"workload": WORKLOAD, "ops_per_step_per_gpu": ops_step,
                       "bytes_per_step_per_gpu": sum(algorithmic_bytes(p[1].shape[1], p[1].shape[0])
                                                     for p in parts),
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"},
            "bit_exact": exact,
            "roofline": {"bound": "hbm", "kernel": "addsub_warp_kernel (4096-bit ops)",
                         "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "peak_source": src,
                         "traffic": read_traffic(), "algorithmic_bytes_per_launch": alg},
            "parts": parts_out,
            "cpu_baseline": cpu,
            "e2e": {"value": round(job_throughput(ops_step, world, e2e_ms), 4), "unit": "Gop/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": round(e2e_ms, 4), "api": "dot_add_host / dot_sub_host"},
            "gpu_launches": 4 * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(data, seconds):
    """The oracle as it stands, on all host cores, over whole steps of the
    workload (or a bounded row sample of it) for about `seconds` seconds."""
    import oracle
    cores = oracle.cores()
    names = ("add_short", "add_long", "sub_short", "sub_long")
    ops_done = 0
    t0 = time.perf_counter()
    reps = 0
    while True:
        for name in names:
            x, y = data[name]
            (oracle.add if name.startswith("add") else oracle.sub)(x, y, threads=cores)
            ops_done += x.shape[0]
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": round(ops_done / dt / 1e9, 6), "unit": "Gop/s", "cores": cores,
            "kind": "oracle", "sample": f"{reps} whole step(s) of the workload, {dt:.1f} s"}


# ----------------------------------------------------------- reference arm
def reference_arm(args, rank, world):
    if rank != 0:
        return
    from paper_2604_21566_gb300 import workloads as W
    import oracle
    # each step: a bounded row sample of both parts, add and sub
    data = W.addsub_bandwidth(short_batch=1 << 17, long_batch=8)
    cores = oracle.cores()
    names = ("add_short", "add_long", "sub_short", "sub_long")

    def step():
        n = 0
        for name in names:
            x, y = data[name]
            (oracle.add if name.startswith("add") else oracle.sub)(x, y, threads=cores)
            n += x.shape[0]
        return n

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    ops = 0
    for _ in range(args.steps):
        ops += step()
    dt = time.perf_counter() - t0
    value = ops / dt / 1e9
    sample = "per step: 2^17 x 4096-bit + 8 x 2^22-bit pairs, add and sub (a row sample of the workload)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gop/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": round(value, 6), "unit": "Gop/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "Gop/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def profile_case(args):
    """Small cases for ncu, a few launches each:
    add  -- dot_add on 2^18 pairs of 4096-bit operands (403 MB, > L2);
    long -- dot_add on 16 pairs of 2^22-bit operands (25 MB, look-back tiles);
    mul  -- dot_mul on 2^16 pairs of 8192-bit operands (256 MB in + out);
    shared -- dot_mul_shared on the tensor cores, 2^16 x 2048-bit (50 MB)."""
    import torch
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    torch.cuda.set_device(0)
    ctx = dot.Context(0)
    if args.case == "shared":
        f, bb = W.shared_operand()
        fd = torch.from_numpy(f.view(np.int32)).cuda()
        b = torch.from_numpy(bb.view(np.int32)).cuda()
        p = torch.empty((bb.shape[0], 128), dtype=torch.int32, device="cuda")
        for _ in range(args.launches):
            dot.mul_shared(fd, b, p, tensor_cores=True, ctx=ctx)
        torch.cuda.synchronize()
        assert ctx.check() == dot.OK
        print("profile case done")
        return
    if args.case == "mul":
        x, y, _ = W.batched_mul(256)
    elif args.case == "long":
        x, y = W.addsub_bandwidth(short_batch=0, long_batch=16)["add_long"]
    else:
        x, y = W.addsub_bandwidth(short_batch=1 << 18, long_batch=0)["add_short"]
    a = torch.from_numpy(x.view(np.int32)).cuda()
    b = torch.from_numpy(y.view(np.int32)).cuda()
    if args.case == "mul":
        p = torch.empty((x.shape[0], 2 * x.shape[1]), dtype=torch.int32, device="cuda")
        for _ in range(args.launches):
            dot.mul(a, b, p, ctx=ctx)
    else:
        s = torch.empty_like(a)
        c = torch.empty(a.shape[0], dtype=torch.int32, device="cuda")
        for _ in range(args.launches):
            dot.add(a, b, out=s, carry=c, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.check() == dot.OK
    print("profile case done")


IMAD_PER_SM_CLK = 64   # 32-bit integer multiply-add lanes per SM per clock (FMA pipe)


def int_peak():
    """Nominal 32-bit IMAD rate (ops/s): SMs x 64 lanes x max SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    try:
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    return sms * IMAD_PER_SM_CLK * mhz * 1e6, sms, mhz


def _event_ms(fn, reps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def suite(args):
    """One JSON line per workload row: correctness mix, batched multiply per
    size, mixed ragged batch vs one launch per size, shared-operand multiply."""
    import torch
    import oracle
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = dot.Context(0)
    peak, sms, mhz = int_peak()

    def dv(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(
            np.int32 if x.dtype == np.uint32 else np.int64)).cuda()

    def hs(t):
        return t.cpu().numpy().view(np.uint32)

    def emit(d):
        d["suite"] = True
        print(json.dumps(d), flush=True)

    def want(name):
        return not args.only or name in args.only.split(",")

    if want("mix"):
        # -- correctness mix: 4096 x 1024-bit, latency-bound
        d = W.correctness_mix()
        a, b = dv(d["x"]), dv(d["y"])
        asub, bsub = dv(d["a_sub"]), dv(d["b_sub"])
        s = torch.empty_like(a)
        c = torch.empty(a.shape[0], dtype=torch.int32, device="cuda")
        p = torch.empty((a.shape[0], 64), dtype=torch.int32, device="cuda")
        t_add = _event_ms(lambda: dot.add(a, b, s, c, ctx=ctx), 200, stream)
        ok = np.array_equal(hs(s), oracle.add(d["x"], d["y"])[0])
        t_sub = _event_ms(lambda: dot.sub(asub, bsub, s, c, ctx=ctx), 200, stream)
        ok &= np.array_equal(hs(s), oracle.sub(d["a_sub"], d["b_sub"])[0])
        t_mul = _event_ms(lambda: dot.mul(a, b, p, ctx=ctx), 200, stream)
        ok &= np.array_equal(hs(p), oracle.mul(d["x"], d["y"], threads=oracle.cores()))
        emit({"workload": "correctness mix: 4096 x 1024-bit (m=32), add/sub/mul", "bit_exact": bool(ok),
              "us_per_call": {"add": round(t_add * 1e3, 2), "sub": round(t_sub * 1e3, 2),
                              "mul": round(t_mul * 1e3, 2)},
              "gop_s": {"add": round(4096 / t_add / 1e6, 3), "sub": round(4096 / t_sub / 1e6, 3),
                        "mul": round(4096 / t_mul / 1e6, 3)}})

    if want("mul"):
        # -- batched multiply at fixed size
        rows = []
        for m in W.BATCHED_MUL_SIZES:
            x, y, _ = W.batched_mul(m)
            a, b = dv(x), dv(y)
            p = torch.empty((x.shape[0], 2 * m), dtype=torch.int32, device="cuda")
            ms = _event_ms(lambda: dot.mul(a, b, p, ctx=ctx), 20, stream)
            sel = np.random.default_rng(m).integers(0, x.shape[0], 512)
            ok = np.array_equal(hs(p)[sel], oracle.mul(x[sel], y[sel]))
            prods = x.shape[0] * m * m
            imad = 2.0 * prods / (ms * 1e-3)
            rows.append({"m_limbs": m, "bits": 32 * m, "ops": x.shape[0], "ms": round(ms, 4),
                         "gop_s": round(x.shape[0] / (ms * 1e-3) / 1e9, 4),
                         "tera_limb_products_s": round(prods / (ms * 1e-3) / 1e12, 3),
                         "GB_s": round(16 * m * x.shape[0] / (ms * 1e-3) / 1e9, 1),
                         "roofline": {"bound": "alu", "achieved_imad_per_s": imad, "peak": peak,
                                      "frac": round(imad / peak, 4)},
                         "bit_exact_sample": bool(ok)})
        emit({"workload": "batched multiply: 2^16 pairs at 256/1024/4096/8192 bits",
              "int_peak": {"imad_per_s": peak, "sms": sms, "sm_mhz": mhz,
                           "per_sm_clk": IMAD_PER_SM_CLK, "algorithmic_imad_per_product": 2},
              "sizes": rows})

    if want("mulx"):
        # -- batched multiply between and above the workload's sizes: one size
        # for each further column shape (12 columns on 16 lanes, 12 on 25, 16)
        rows = []
        for m in (192, 300, 512):
            x, y, _ = W.batched_mul(m)
            a, b = dv(x), dv(y)
            p = torch.empty((x.shape[0], 2 * m), dtype=torch.int32, device="cuda")
            ms = _event_ms(lambda: dot.mul(a, b, p, ctx=ctx), 20, stream)
            sel = np.random.default_rng(m).integers(0, x.shape[0], 256)
            ok = np.array_equal(hs(p)[sel], oracle.mul(x[sel], y[sel], threads=oracle.cores()))
            prods = x.shape[0] * m * m
            imad = 2.0 * prods / (ms * 1e-3)
            rows.append({"m_limbs": m, "bits": 32 * m, "ops": x.shape[0], "ms": round(ms, 4),
                         "cols_per_lane": dot.plan(dot.OP_MUL, m, x.shape[0]).seg_limbs,
                         "tera_limb_products_s": round(prods / (ms * 1e-3) / 1e12, 3),
                         "roofline": {"bound": "alu", "achieved_imad_per_s": imad, "peak": peak,
                                      "frac": round(imad / peak, 4)},
                         "bit_exact_sample": bool(ok)})
        emit({"workload": "batched multiply: 2^16 pairs at 6144/9600/16384 bits", "sizes": rows})

    if want("sqr"):
        # -- batched square (half the partial products) vs the general product
        rows = []
        for m in (32, 128, 256):
            x, _, _ = W.batched_mul(m)
            a = dv(x)
            p = torch.empty((x.shape[0], 2 * m), dtype=torch.int32, device="cuda")
            t_mul = _event_ms(lambda: dot.mul(a, a, p, ctx=ctx), 20, stream)
            t_sqr = _event_ms(lambda: dot.sqr(a, p, ctx=ctx), 20, stream)
            sel = np.random.default_rng(m).integers(0, x.shape[0], 512)
            ok = np.array_equal(hs(p)[sel], oracle.sqr(x[sel]))
            rows.append({"m_limbs": m, "ops": x.shape[0], "ms_mul": round(t_mul, 4), "ms_sqr": round(t_sqr, 4),
                         "speedup_sqr_vs_mul": round(t_mul / t_sqr, 3), "bit_exact_sample": bool(ok)})
        emit({"workload": "batched square: 2^16 operands at 1024/4096/8192 bits", "sizes": rows})

    if want("kara"):
        # -- Karatsuba above the base case: effective schoolbook limb products per second
        rows = []
        for m, batch in ((1024, 4096), (2048, 2048), (4096, 1024), (8192, 256)):
            g = np.random.default_rng(5000 + m)
            x = g.integers(0, 2 ** 32, (batch, m), dtype=np.uint64).astype(np.uint32)
            y = g.integers(0, 2 ** 32, (batch, m), dtype=np.uint64).astype(np.uint32)
            a, b = dv(x), dv(y)
            p = torch.empty((batch, 2 * m), dtype=torch.int32, device="cuda")
            ms = _event_ms(lambda: dot.mul_karatsuba(a, b, p, ctx=ctx), 5, stream)
            sel = np.arange(0, batch, max(1, batch // 4))
            ok = np.array_equal(hs(p)[sel], oracle.mul(x[sel], y[sel], threads=8))
            prods = batch * m * m
            rows.append({"m_limbs": m, "bits": 32 * m, "ops": batch, "ms": round(ms, 4),
                         "gop_s": round(batch / (ms * 1e-3) / 1e9, 6),
                         "schoolbook_equiv_tera_products_s": round(prods / (ms * 1e-3) / 1e12, 3),
                         "bit_exact_sample": bool(ok)})
        emit({"workload": "Karatsuba above 512 limbs: 32k..262k-bit products",
              "note": "schoolbook-equivalent rate = batch m^2 / time (m^2 products a schoolbook would do)",
              "sizes": rows})

    if want("mixed"):
        # -- mixed ragged batch: one persistent bucketed kernel vs one launch per size
        w = W.ragged_mixed()
        n = w["op"].size
        desc = np.zeros(n, dtype=[("op", "<u4"), ("m", "<u4"), ("a_off", "<u8"), ("b_off", "<u8"),
                                  ("r_off", "<u8")])
        desc["op"], desc["m"] = w["op"], w["m"]
        desc["a_off"] = desc["b_off"] = w["a_off"][:-1]
        desc["r_off"] = w["r_off"][:-1]
        ddesc = torch.from_numpy(desc.view(np.uint8).copy()).cuda()
        a, b = dv(w["a"]), dv(w["b"])
        r = torch.zeros(int(w["r_off"][-1]), dtype=torch.int32, device="cuda")
        cr = torch.zeros(n, dtype=torch.int32, device="cuda")
        t_mixed = _event_ms(lambda: dot.mixed_ragged(ddesc, a, b, r, cr, ctx=ctx), 20, stream)
        wr, wc = oracle.mixed(desc["op"], desc["m"], desc["a_off"], desc["b_off"], desc["r_off"],
                              w["a"], w["b"], w["r_off"][-1])
        ok = np.array_equal(hs(r), wr) and np.array_equal(hs(cr), wc)
        # one launch per (op, size): operands regrouped contiguously beforehand
        groups = []
        for opc in (W.OP_ADD, W.OP_SUB, W.OP_MUL):
            for m in np.unique(w["m"][w["op"] == opc]):
                idx = np.nonzero((w["op"] == opc) & (w["m"] == m))[0]
                rows_a = np.stack([w["a"][int(w["a_off"][i]):int(w["a_off"][i]) + m] for i in idx])
                rows_b = np.stack([w["b"][int(w["a_off"][i]):int(w["a_off"][i]) + m] for i in idx])
                ga, gb = dv(rows_a), dv(rows_b)
                out = torch.empty((idx.size, 2 * m if opc == W.OP_MUL else m), dtype=torch.int32,
                                  device="cuda")
                gc = torch.empty(idx.size, dtype=torch.int32, device="cuda")
                groups.append((opc, ga, gb, out, gc))

        def per_size():
            for opc, ga, gb, out, gc in groups:
                if opc == W.OP_MUL:
                    dot.mul(ga, gb, out, ctx=ctx)
                elif opc == W.OP_ADD:
                    dot.add(ga, gb, out, gc, ctx=ctx)
                else:
                    dot.sub(ga, gb, out, gc, ctx=ctx)
        t_per = _event_ms(per_size, 5, stream)
        prods = int((w["m"][w["op"] == W.OP_MUL].astype(np.int64) ** 2).sum())
        emit({"workload": "ragged mixed: 200k ops, 30/30/40 add/sub/mul, 128..16384 bits",
              "bit_exact": bool(ok), "ms_persistent_graph": round(t_mixed, 4),
              "gop_s": round(n / (t_mixed * 1e-3) / 1e9, 4),
              "ms_one_launch_per_size": round(t_per, 4), "launches_per_size": len(groups),
              "speedup_vs_per_size": round(t_per / t_mixed, 3),
              "roofline": {"bound": "alu", "achieved_imad_per_s": 2.0 * prods / (t_mixed * 1e-3),
                           "peak": peak, "frac": round(2.0 * prods / (t_mixed * 1e-3) / peak, 4)}})

    if want("shared"):
        # -- shared operand: Toeplitz product on the tensor cores vs the INT32 paths
        f, bb = W.shared_operand()
        n = bb.shape[0]
        a = dv(np.ascontiguousarray(np.broadcast_to(f, bb.shape)))
        fd, b = dv(f), dv(bb)
        p = torch.empty((n, 128), dtype=torch.int32, device="cuda")
        sel = np.arange(0, n, 97)
        want = oracle.mul(np.broadcast_to(f, (sel.size, 64)), bb[sel])
        t_int = _event_ms(lambda: dot.mul(a, b, p, ctx=ctx), 50, stream)
        ok = np.array_equal(hs(p)[sel], want)
        t_int_sh = _event_ms(lambda: dot.mul_shared(fd, b, p, tensor_cores=False, ctx=ctx), 50, stream)
        ok &= np.array_equal(hs(p)[sel], want)
        t_tc = _event_ms(lambda: dot.mul_shared(fd, b, p, tensor_cores=True, ctx=ctx), 50, stream)
        ok &= np.array_equal(hs(p)[sel], want)
        # tensor work issued: 48 MMAs of 128 x 128 x 16 per 128 operands
        flops = 2.0 * 128 * 128 * 16 * 48 * ((n + 127) // 128)
        useful = 2.0 * 256 * 256 * n
        hbm, _ = peaks()
        tc_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
        bytes_moved = n * (256 + 512) + 256
        emit({"workload": "shared operand: fixed 2048-bit x 2^16 2048-bit", "bit_exact_sample": bool(ok),
              "ms_int32_batched": round(t_int, 4), "ms_int32_shared": round(t_int_sh, 4),
              "ms_tensor": round(t_tc, 4), "speedup_tensor_vs_int32": round(t_int / t_tc, 3),
              "gop_s_tensor": round(n / (t_tc * 1e-3) / 1e9, 4),
              "roofline_tensor": {"issued_tflop_s": round(flops / (t_tc * 1e-3) / 1e12, 1),
                                  "useful_tflop_s": round(useful / (t_tc * 1e-3) / 1e12, 1),
                                  "peak_fp16_tflop_s": tc_peak,
                                  "frac_issued": round(flops / (t_tc * 1e-3) / 1e12 / tc_peak, 4),
                                  "GB_s": round(bytes_moved / (t_tc * 1e-3) / 1e9, 1),
                                  "frac_hbm": round(bytes_moved / (t_tc * 1e-3) / 1e9 / hbm, 4)}})
    assert ctx.check() == dot.OK
    ctx.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--suite", action="store_true",
                    help="measure every workload row (one JSON line each) instead of the bench step")
    ap.add_argument("--profile-case", action="store_true",
                    help="run only the small ncu case of the dominant kernel")
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--only", default="", help="--suite rows to run: mix,mul,mulx,sqr,kara,mixed,shared")
    ap.add_argument("--case", choices=["add", "long", "mul", "shared"], default="add",
                    help="which kernel --profile-case runs")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["dot", "reference"], default="dot")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_info()
    if args.profile_case or args.suite:
        from paper_2604_21566_gb300 import build as B
        B.build()
        (suite if args.suite else profile_case)(args)
        return
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    from paper_2604_21566_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        # other ranks wait for rank 0's build of the shared in-tree library
        lib = os.path.join(ROOT, "paper_2604_21566_gb300", "libdot.so")
        t0 = time.time()
        while not os.path.exists(lib) and time.time() - t0 < 600:
            time.sleep(1)
    gpu_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
