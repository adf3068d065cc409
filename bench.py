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

The same line carries ``rows``: the other workloads -- the correctness mix
(4096 x 1024-bit add, sub, mul), the batched multiply (2^16 pairs at 256 to
8192 bits), the 200k-op ragged mixed batch (graph replay vs one launch per
size) and the shared-operand product (tensor cores vs INT32) -- each timed
call by call with L2 flushed before it, checked on every row against the
oracle, reported against a measured peak (HBM copy and bf16 GEMM from
MEASURED_PEAKS.json; integer-pipe ceilings from the libdotprobe
microbenchmarks run in the same process), with the oracle's all-core time on
the same rows and the clocks seen meanwhile.

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
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary: (read + write, read, write), or Nones if the summary is missing
    or was taken on different kernel sources."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None, None, None
    vals = {}
    for ln in text.splitlines():
        if ":" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None, None, None
    try:
        rd, wr = int(vals["dram_read_bytes_per_launch"]), int(vals["dram_write_bytes_per_launch"])
    except (KeyError, ValueError):
        return None, None, None
    return rd + wr, rd, wr


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

    rows = None
    if rank == 0 and not args.no_rows:
        rows = workload_rows(ctx, stream, local)
    if world > 1:
        torch.distributed.barrier()

    if rank == 0:
        hbm, src = peaks()
        dom = "add_short"
        dom_ms = 0.5 * (per_launch["add_short"] + per_launch["sub_short"])
        x, _ = data[dom]
        alg = algorithmic_bytes(x.shape[1], x.shape[0])
        traffic, traffic_rd, traffic_wr = read_traffic()
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
                         "traffic": traffic, "traffic_read": traffic_rd, "traffic_write": traffic_wr,
                         "traffic_source": "ncu dram__bytes_read.sum / dram__bytes_write.sum of one "
                                           "launch that follows an identical launch (its writes include "
                                           "the evictions of the previous launch's dirty lines), "
                                           "scaled from 2^18 to the bench's 2^20 pairs",
                         "algorithmic_bytes_per_launch": alg,
                         "algorithmic_read_bytes_per_launch": x.shape[0] * 8 * x.shape[1]},
            "parts": parts_out,
            "cpu_baseline": cpu,
            "e2e": {"value": round(job_throughput(ops_step, world, e2e_ms), 4), "unit": "Gop/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": round(e2e_ms, 4), "api": "dot_add_host / dot_sub_host"},
            "gpu_launches": 4 * args.steps,
            "clocks": clocks,
            "rows": rows,
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
    # each step: one whole step of the workload (add and sub of both parts),
    # the same rows and calls as the GPU arm's cpu_baseline; about 30 ms on 16
    # host cores
    data = W.addsub_bandwidth()
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
    sample = "per step: the whole workload (2^20 x 4096-bit + 64 x 2^22-bit pairs, add and sub)"
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
    long -- dot_add on 64 pairs of 2^22-bit operands (100 MB, look-back tiles:
            the bench's own part, at the bench's grid);
    mul  -- dot_mul on 2^16 pairs of 8192-bit operands (256 MB in + out);
    shared -- dot_mul_shared on the tensor cores, 2^16 x 2048-bit (50 MB);
    shared2p18 -- the same on 2^18 operands (201 MB, > L2, so that the DRAM
            counters see the products written);
    shared128 -- the same at 4096 bits (two K slices, 100 MB);
    mixed -- dot_mixed_ragged on 20k ops of the mixed-batch recipe (graph
            replay: classify, plan, scatter, then the product and add/sub
            kernels)."""
    import torch
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    torch.cuda.set_device(0)
    ctx = dot.Context(0)
    if args.case == "mixed":
        w = W.ragged_mixed(nops=20_000)
        ddesc = torch.from_numpy(ragged_descriptors(w).view(np.uint8).copy()).cuda()
        a, b = _dv(w["a"]), _dv(w["b"])
        r = torch.zeros(int(w["r_off"][-1]), dtype=torch.int32, device="cuda")
        cr = torch.zeros(w["op"].size, dtype=torch.int32, device="cuda")
        for _ in range(args.launches):
            dot.mixed_ragged(ddesc, a, b, r, cr, ctx=ctx)
        torch.cuda.synchronize()
        assert ctx.check() == dot.OK
        print("profile case done")
        return
    if args.case in ("shared", "shared2p18", "shared128"):
        f, bb = W.shared_operand(m=128 if args.case == "shared128" else 64,
                                 batch=1 << (18 if args.case == "shared2p18" else 16))
        fd = torch.from_numpy(f.view(np.int32)).cuda()
        b = torch.from_numpy(bb.view(np.int32)).cuda()
        p = torch.empty((bb.shape[0], 2 * bb.shape[1]), dtype=torch.int32, device="cuda")
        for _ in range(args.launches):
            dot.mul_shared(fd, b, p, tensor_cores=True, ctx=ctx)
        torch.cuda.synchronize()
        assert ctx.check() == dot.OK
        print("profile case done")
        return
    if args.case == "mul":
        x, y, _ = W.batched_mul(256)
    elif args.case == "long":
        x, y = W.addsub_bandwidth(short_batch=0, long_batch=64)["add_long"]
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


# ------------------------------------------------------------ workload rows
# Every row below times its calls one by one with CUDA events on the calling
# stream after writing a 256 MB buffer (twice the L2) on that stream and then
# reading it back, so no call finds its inputs in L2 and none pays for writing
# back the flush's dirty lines; checks every result against the oracle; and
# times the oracle on all host cores on the same rows as the CPU baseline.
L2_FLUSH_BYTES = 256 << 20
L2_NOTE = "flushed before each timed call (256 MB written, then read back)"
UNSATURATED_DIGIT_BITS = 27   # largest digit whose 64-bit column sums need no carry up to 512 limbs


def measured_peaks():
    """HBM GB/s and dense bf16 TF/s (burst) from MEASURED_PEAKS.json, else the fallback figures."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class Timer:
    """Cold-L2 CUDA-event timing of single calls on one stream."""

    def __init__(self, stream):
        import torch
        self.stream = stream
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def ms(self, fn, reps, warm=3):
        import torch
        for _ in range(warm):
            fn()
        ev = []
        for _ in range(reps):
            self.flush.zero_()
            self.flush.sum()   # leaves L2 holding clean lines of the flush buffer
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            fn()
            e1.record(self.stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        t = [a.elapsed_time(b) for a, b in ev]
        return statistics.mean(t), statistics.median(t)


def _cpu(fn, units, unit, sample):
    """Time one oracle call on all host cores: (result, cpu_baseline dict)."""
    import oracle
    t0 = time.perf_counter()
    res = fn(oracle.cores())
    dt = time.perf_counter() - t0
    return res, {"value": round(units / dt / 1e9, 6), "unit": unit, "cores": oracle.cores(), "kind": "oracle",
                 "sample": sample, "seconds": round(dt, 3)}


def _dv(x):
    import torch
    x = np.ascontiguousarray(x)
    return torch.from_numpy(x.view(np.int32 if x.dtype == np.uint32 else np.int64)).cuda()


def _hs(t):
    return t.cpu().numpy().view(np.uint32)


def row_peaks():
    """Integer-pipe ceilings and tensor-pipe shape rates measured on this GPU
    (libdotprobe)."""
    from paper_2604_21566_gb300 import probe
    return probe.measure()


def _int_roofline(products, ms, pk):
    pair = pk["mul_pair"]["per_s"]
    mix = pk["colsum_r8"]["per_s"]
    rate = products / (ms * 1e-3)
    return {"bound": "alu", "achieved_products_per_s": round(rate, 1), "unit": "limb products/s",
            "peak": round(pair, 1), "frac": round(rate / pair, 4),
            "peak_source": "measured: mul.lo + mul.hi pair probe (libdotprobe)",
            "peak_colsum_mix": round(mix, 1), "frac_of_colsum_mix": round(rate / mix, 4)}


def row_c1(ctx, timer, pk, reps=100):
    """Correctness mix: 4096 x 1024-bit add, sub and mul."""
    import oracle
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    import torch
    hbm, _, src = measured_peaks()
    d = W.correctness_mix()
    n, m = d["x"].shape
    a, b = _dv(d["x"]), _dv(d["y"])
    asub, bsub = _dv(d["a_sub"]), _dv(d["b_sub"])
    s = torch.empty_like(a)
    c = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty((n, 2 * m), dtype=torch.int32, device="cuda")
    floor = pk["launch_floor"]["us"]
    out = {"workload": "4096 x 1024-bit pairs (m = 32): 50% uniform, 25% full-ripple all-ones, 25% sparse",
           "l2": L2_NOTE, "ops": {}}
    exact = True
    cpu = {}
    for name in ("add", "sub", "mul"):
        if name == "add":
            fn, x, y = (lambda: dot.add(a, b, s, c, ctx=ctx)), d["x"], d["y"]
        elif name == "sub":
            fn, x, y = (lambda: dot.sub(asub, bsub, s, c, ctx=ctx)), d["a_sub"], d["b_sub"]
        else:
            fn, x, y = (lambda: dot.mul(a, b, p, ctx=ctx)), d["x"], d["y"]
        mean, med = timer.ms(fn, reps)
        if name == "mul":
            want, cpu[name] = _cpu(lambda t: oracle.mul(x, y, threads=t), n, "Gop/s", "all 4096 rows")
            exact &= bool(np.array_equal(_hs(p), want))
            roof = _int_roofline(n * m * m, mean, pk)
        else:
            f = oracle.add if name == "add" else oracle.sub
            (ws, wc), cpu[name] = _cpu(lambda t: f(x, y, threads=t), n, "Gop/s", "all 4096 rows")
            exact &= bool(np.array_equal(_hs(s), ws) and np.array_equal(_hs(c), wc))
            gbs = n * (12 * m + 4) / (mean * 1e-3) / 1e9
            roof = {"bound": "latency", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(gbs / hbm, 4), "peak_source": src,
                    "launch_floor_us": floor, "frac_of_launch_floor": round(floor / (mean * 1e3), 4)}
        out["ops"][name] = {"us": round(mean * 1e3, 2), "us_median": round(med * 1e3, 2),
                            "gop_s": round(n / (mean * 1e-3) / 1e9, 4), "roofline": roof}
    out["bit_exact"] = exact
    out["bit_exact_rows"] = "all"
    out["cpu_baseline"] = cpu
    return out


def row_c3(ctx, timer, pk, reps=20):
    """Batched multiply at fixed size: 2^16 pairs at 256, 1024, 4096, 8192 bits."""
    import oracle
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    import torch
    hbm, _, src = measured_peaks()
    sizes = {}
    exact = True
    for m in W.BATCHED_MUL_SIZES:
        x, y, _ = W.batched_mul(m)
        n = x.shape[0]
        a, b = _dv(x), _dv(y)
        p = torch.empty((n, 2 * m), dtype=torch.int32, device="cuda")
        mean, med = timer.ms(lambda: dot.mul(a, b, p, ctx=ctx), reps)
        want, cpu = _cpu(lambda t: oracle.mul(x, y, threads=t), n, "Gop/s", f"all {n} rows")
        ok = bool(np.array_equal(_hs(p), want))
        exact &= ok
        roof = _int_roofline(n * m * m, mean, pk)
        gbs = n * 16 * m / (mean * 1e-3) / 1e9
        roof["achieved_GB_s"] = round(gbs, 1)
        roof["frac_hbm"] = round(gbs / hbm, 4)
        roof["hbm_peak_source"] = src
        if m <= 8:
            roof["bound"] = "latency (too little work per launch for either pipe)"
        sizes[f"{32 * m}_bit"] = {"m_limbs": m, "ops": n, "ms": round(mean, 4), "ms_median": round(med, 4),
                                  "gop_s": round(n / (mean * 1e-3) / 1e9, 4),
                                  "kernel": ("one product per thread" if dot.plan(dot.OP_MUL, m, n).kernel == 4
                                             else f"column sums, {dot.plan(dot.OP_MUL, m, n).seg_limbs} columns per lane"),
                                  "roofline": roof, "bit_exact": ok, "cpu_baseline": cpu}
        del a, b, p
    return {"workload": "2^16 pairs at 256/1024/4096/8192 bits, uniform limbs + 10% both-all-ones pairs",
            "l2": L2_NOTE, "bit_exact": exact, "bit_exact_rows": "all",
            "sizes": sizes}


def ragged_descriptors(w):
    desc = np.zeros(w["op"].size, dtype=[("op", "<u4"), ("m", "<u4"), ("a_off", "<u8"), ("b_off", "<u8"),
                                         ("r_off", "<u8")])
    desc["op"], desc["m"] = w["op"], w["m"]
    desc["a_off"] = desc["b_off"] = w["a_off"][:-1]
    desc["r_off"] = w["r_off"][:-1]
    return desc


def row_c4(ctx, timer, pk, reps=10):
    """Ragged mixed batch: one persistent bucketed kernel from a CUDA graph vs
    one launch per (op, size)."""
    import oracle
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    import torch
    w = W.ragged_mixed()
    n = w["op"].size
    desc = ragged_descriptors(w)
    ddesc = torch.from_numpy(desc.view(np.uint8).copy()).cuda()
    a, b = _dv(w["a"]), _dv(w["b"])
    r = torch.zeros(int(w["r_off"][-1]), dtype=torch.int32, device="cuda")
    cr = torch.zeros(n, dtype=torch.int32, device="cuda")
    mean, med = timer.ms(lambda: dot.mixed_ragged(ddesc, a, b, r, cr, ctx=ctx), reps)
    (wr, wc), cpu = _cpu(lambda t: oracle.mixed(desc["op"], desc["m"], desc["a_off"], desc["b_off"],
                                                desc["r_off"], w["a"], w["b"], w["r_off"][-1], threads=t),
                         n, "Gop/s", f"all {n} ops")
    exact = bool(np.array_equal(_hs(r), wr) and np.array_equal(_hs(cr), wc))
    # one launch per (op, size): operands regrouped contiguously beforehand
    groups = []
    for opc in (W.OP_ADD, W.OP_SUB, W.OP_MUL):
        for m in np.unique(w["m"][w["op"] == opc]):
            idx = np.nonzero((w["op"] == opc) & (w["m"] == m))[0]
            lo = w["a_off"][idx].astype(np.int64)
            sel = (lo[:, None] + np.arange(m)[None, :]).reshape(-1)
            ga, gb = _dv(w["a"][sel].reshape(idx.size, m)), _dv(w["b"][sel].reshape(idx.size, m))
            outw = 2 * m if opc == W.OP_MUL else m
            groups.append((opc, ga, gb, torch.empty((idx.size, outw), dtype=torch.int32, device="cuda"),
                           torch.empty(idx.size, dtype=torch.int32, device="cuda")))

    def per_size():
        for opc, ga, gb, go, gc in groups:
            if opc == W.OP_MUL:
                dot.mul(ga, gb, go, ctx=ctx)
            elif opc == W.OP_ADD:
                dot.add(ga, gb, go, gc, ctx=ctx)
            else:
                dot.sub(ga, gb, go, gc, ctx=ctx)
    t_per, _ = timer.ms(per_size, 3, warm=1)
    mulm = w["m"][w["op"] == W.OP_MUL].astype(np.int64)
    prods = int((mulm ** 2).sum())
    roof = _int_roofline(prods, mean, pk)
    return {"workload": "200k ops, 30/30/40 add/sub/mul, log-uniform 128..16384 bits, shuffled",
            "l2": L2_NOTE, "bit_exact": exact, "bit_exact_rows": "all",
            "ms_persistent_graph": round(mean, 4), "ms_median": round(med, 4),
            "gop_s": round(n / (mean * 1e-3) / 1e9, 4),
            "ms_one_launch_per_size": round(t_per, 4), "launches_per_size": len(groups),
            "speedup_vs_per_size": round(t_per / mean, 3), "mul_limb_products": prods,
            "roofline": roof, "cpu_baseline": cpu}


def row_n4(ctx, timer, pk, reps=10):
    """Unsaturated radix (27-bit digits, one mad.wide per digit product, no
    carry chain) against the saturated 32-bit-limb multiply, at equal bit
    sizes: 2^16 products each."""
    import oracle
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    import torch
    out = {"workload": "2^16 pairs at 4096 and 8192 bits: radix 2^27 digits (dot_mul_unsat) vs "
                       "radix 2^32 limbs (dot_mul)", "l2": L2_NOTE, "sizes": {}}
    exact = True
    madw = pk["madwide_r8"]["per_s"]
    for bits_total in (4096, 8192):
        x, y = W.unsaturated_mul(bits_total)
        nb, n = x.shape
        a, b = _dv(x), _dv(y)
        p = torch.empty((nb, 2 * n), dtype=torch.int32, device="cuda")
        t_unsat, _ = timer.ms(lambda: dot.mul_unsat(a, b, p, ctx=ctx), reps)
        want, cpu = _cpu(lambda t: oracle.mul_radix(x, y, W.UNSAT_BITS, threads=t), nb, "Gop/s", f"all {nb} rows")
        ok = bool(np.array_equal(_hs(p), want))
        exact &= ok
        xs, ys, _ = W.batched_mul(bits_total // 32)
        m = xs.shape[1]
        a2, b2 = _dv(xs), _dv(ys)
        p2 = torch.empty((nb, 2 * m), dtype=torch.int32, device="cuda")
        t_sat, _ = timer.ms(lambda: dot.mul(a2, b2, p2, ctx=ctx), reps)
        rate = nb * n * n / (t_unsat * 1e-3)
        out["sizes"][f"{bits_total}_bit"] = {
            "digits": n, "limbs": m, "ms_unsat": round(t_unsat, 4), "ms_saturated": round(t_sat, 4),
            "unsat_time_vs_saturated": round(t_unsat / t_sat, 3), "bit_exact": ok,
            "roofline": {"bound": "alu", "achieved": round(rate, 1), "unit": "digit products/s",
                         "peak": round(madw, 1), "frac": round(rate / madw, 4),
                         "peak_source": "measured: mad.wide.u32 column-sum probe (libdotprobe)"},
            "cpu_baseline": cpu}
        del a, b, p, a2, b2, p2
    out["bit_exact"] = exact
    out["bit_exact_rows"] = "all"
    return out


def tz_units_per_tile(m: int) -> int:
    """128 x 128 x 16 MMA units the Toeplitz kernel issues per tile of 128
    operands: per 128-column output block, one rank-one bias product per K
    slice and 8 k-steps for every 128-digit k-block that meets the block (the
    issuer's own loop).  m = 64: 4 + 48 = 52; m = 128: 16 + 160 = 176."""
    kb_n = (4 * m + 127) // 128
    cb_n = (8 * m + 127) // 128
    slices = 1 if m <= 64 else 2
    units = slices * cb_n
    for cb in range(cb_n):
        units += 8 * (min(kb_n - 1, cb) - max(0, cb - kb_n) + 1)
    return units


def _tc_shape(pk, m, tflops):
    """The kernel's own product shape issued back to back alone (libdotprobe):
    M = 128, N = 128, K = 16 with A from tensor memory (up to 64 limbs) or
    shared memory (two K slices); the widest single-CTA shape beside it."""
    key = "mma_n128_tmem" if m <= 64 else "mma_n128_smem"
    shape = pk[key]["per_s"] / 1e12
    widest = pk["mma_n256_tmem"]["per_s"] / 1e12
    return {"peak_own_shape": round(shape, 1), "own_shape": key, "frac_of_own_shape": round(tflops / shape, 4),
            "peak_n256_tmem": round(widest, 1)}


def row_c5(ctx, timer, pk, reps=50):
    """Shared operand: one fixed 2048-bit multiplier x 2^16 2048-bit operands,
    Toeplitz product on the tensor cores vs the INT32 paths."""
    import oracle
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    import torch
    hbm, tc_peak, src = measured_peaks()
    f, bb = W.shared_operand()
    n, m = bb.shape
    fa = np.ascontiguousarray(np.broadcast_to(f, bb.shape))
    a, fd, b = _dv(fa), _dv(f), _dv(bb)
    p = torch.empty((n, 2 * m), dtype=torch.int32, device="cuda")
    want, cpu = _cpu(lambda t: oracle.mul(fa, bb, threads=t), n, "Gop/s", f"all {n} rows")
    t_int, _ = timer.ms(lambda: dot.mul(a, b, p, ctx=ctx), reps)
    ok = bool(np.array_equal(_hs(p), want))
    t_sh, _ = timer.ms(lambda: dot.mul_shared(fd, b, p, tensor_cores=False, ctx=ctx), reps)
    ok &= bool(np.array_equal(_hs(p), want))
    t_tc, med = timer.ms(lambda: dot.mul_shared(fd, b, p, tensor_cores=True, ctx=ctx), reps)
    ok &= bool(np.array_equal(_hs(p), want))
    tiles = (n + 127) // 128
    issued = 2.0 * 128 * 128 * 16 * tz_units_per_tile(m) * tiles
    useful = 2.0 * (4 * m) ** 2 * n
    bytes_moved = n * 12 * m + 4 * m
    tflops = issued / (t_tc * 1e-3) / 1e12
    return {"workload": "fixed 2048-bit x 2^16 2048-bit (m = 64), uniform limbs",
            "l2": L2_NOTE, "bit_exact": ok, "bit_exact_rows": "all",
            "ms_tensor": round(t_tc, 4), "ms_tensor_median": round(med, 4), "ms_int32_batched": round(t_int, 4),
            "ms_int32_shared": round(t_sh, 4), "speedup_tensor_vs_int32": round(t_int / t_tc, 3),
            "gop_s_tensor": round(n / (t_tc * 1e-3) / 1e9, 4),
            "roofline": {"bound": "tensor", "achieved": round(tflops, 1), "peak": tc_peak, "unit": "TFLOP/s",
                         "frac": round(tflops / tc_peak, 4),
                         "peak_source": f"{src} bf16 burst (fp16 runs at the bf16 rate)",
                         "issued_units_128x128x16_per_tile": tz_units_per_tile(m),
                         "useful_tflop_s": round(useful / (t_tc * 1e-3) / 1e12, 1),
                         "frac_useful": round(useful / (t_tc * 1e-3) / 1e12 / tc_peak, 4),
                         "achieved_GB_s": round(bytes_moved / (t_tc * 1e-3) / 1e9, 1),
                         "frac_hbm": round(bytes_moved / (t_tc * 1e-3) / 1e9 / hbm, 4),
                         **_tc_shape(pk, m, tflops)},
            "int32_roofline": _int_roofline(n * m * m, t_int, pk),
            "cpu_baseline": cpu}


def row_n3(ctx, timer, pk, reps=20):
    """Split-K tensor path: one fixed 4096-bit multiplier x 2^16 4096-bit
    operands (two K slices of 256 digits) vs the INT32 shared-operand path."""
    import oracle
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    import torch
    hbm, tc_peak, src = measured_peaks()
    f, bb = W.shared_operand(m=128)
    n, m = bb.shape
    fa = np.ascontiguousarray(np.broadcast_to(f, bb.shape))
    fd, b = _dv(f), _dv(bb)
    p = torch.empty((n, 2 * m), dtype=torch.int32, device="cuda")
    want, cpu = _cpu(lambda t: oracle.mul(fa, bb, threads=t), n, "Gop/s", f"all {n} rows")
    t_sh, _ = timer.ms(lambda: dot.mul_shared(fd, b, p, tensor_cores=False, ctx=ctx), reps)
    ok = bool(np.array_equal(_hs(p), want))
    t_tc, med = timer.ms(lambda: dot.mul_shared(fd, b, p, tensor_cores=True, ctx=ctx), reps)
    ok &= bool(np.array_equal(_hs(p), want))
    tiles = (n + 127) // 128
    issued = 2.0 * 128 * 128 * 16 * tz_units_per_tile(m) * tiles
    useful = 2.0 * (4 * m) ** 2 * n
    tflops = issued / (t_tc * 1e-3) / 1e12
    return {"workload": "fixed 4096-bit x 2^16 4096-bit (m = 128, two K slices)", "l2": L2_NOTE,
            "bit_exact": ok, "bit_exact_rows": "all", "ms_tensor": round(t_tc, 4),
            "ms_tensor_median": round(med, 4), "ms_int32_shared": round(t_sh, 4),
            "speedup_tensor_vs_int32": round(t_sh / t_tc, 3),
            "roofline": {"bound": "tensor", "achieved": round(tflops, 1), "peak": tc_peak, "unit": "TFLOP/s",
                         "frac": round(tflops / tc_peak, 4),
                         "peak_source": f"{src} bf16 burst (fp16 runs at the bf16 rate)",
                         "issued_units_128x128x16_per_tile": tz_units_per_tile(m),
                         "useful_tflop_s": round(useful / (t_tc * 1e-3) / 1e12, 1),
                         "frac_useful": round(useful / (t_tc * 1e-3) / 1e12 / tc_peak, 4),
                         **_tc_shape(pk, m, tflops)},
            "int32_roofline": _int_roofline(n * m * m, t_sh, pk), "cpu_baseline": cpu}


def workload_rows(ctx, stream, local):
    """The correctness-mix, batched-multiply, mixed-batch and shared-operand
    rows of the default bench line, with the clocks seen while they ran."""
    sampler = ClockSampler(local)
    sampler.start()
    timer = Timer(stream)
    pk = row_peaks()
    rows = {"int_peaks": pk,
            "C1_correctness_mix": row_c1(ctx, timer, pk),
            "C3_batched_mul": row_c3(ctx, timer, pk),
            "C4_ragged_mixed": row_c4(ctx, timer, pk),
            "C5_shared_operand": row_c5(ctx, timer, pk),
            "N3_split_k_tensor": row_n3(ctx, timer, pk),
            "N4_unsaturated_radix": row_n4(ctx, timer, pk)}
    rows["clocks"] = sampler.stop()
    return rows


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
    """One JSON line per row: the driver line's rows, then the further rows
    (multiply at other sizes, squares, Karatsuba)."""
    import torch
    import oracle
    from paper_2604_21566_gb300 import dot
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = dot.Context(0)
    timer = Timer(stream)
    pk = row_peaks()

    def emit(name, d):
        print(json.dumps({"suite": name, **d}), flush=True)

    def want(name):
        return not args.only or name in args.only.split(",")

    emit("int_peaks", pk)
    if want("mix"):
        emit("C1_correctness_mix", row_c1(ctx, timer, pk))
    if want("mul"):
        emit("C3_batched_mul", row_c3(ctx, timer, pk))
    if want("mixed"):
        emit("C4_ragged_mixed", row_c4(ctx, timer, pk))
    if want("shared"):
        emit("C5_shared_operand", row_c5(ctx, timer, pk))
    if want("splitk"):
        emit("N3_split_k_tensor", row_n3(ctx, timer, pk))
    if want("unsat"):
        emit("N4_unsaturated_radix", row_n4(ctx, timer, pk))
    if want("mulx"):
        # batched multiply between and above the workload's sizes: one size
        # for each further column shape (12 columns on 16 lanes, 12 on 25, 16)
        from paper_2604_21566_gb300 import workloads as W
        rows = []
        for m in (192, 300, 512):
            x, y, _ = W.batched_mul(m)
            a, b = _dv(x), _dv(y)
            p = torch.empty((x.shape[0], 2 * m), dtype=torch.int32, device="cuda")
            ms, _ = timer.ms(lambda: dot.mul(a, b, p, ctx=ctx), 10)
            sel = np.random.default_rng(m).integers(0, x.shape[0], 256)
            ok = np.array_equal(_hs(p)[sel], oracle.mul(x[sel], y[sel], threads=oracle.cores()))
            rows.append({"m_limbs": m, "bits": 32 * m, "ops": x.shape[0], "ms": round(ms, 4),
                         "cols_per_lane": dot.plan(dot.OP_MUL, m, x.shape[0]).seg_limbs,
                         "roofline": _int_roofline(x.shape[0] * m * m, ms, pk), "bit_exact_sample": bool(ok)})
        emit("batched_mul_other_sizes", {"workload": "2^16 pairs at 6144/9600/16384 bits", "sizes": rows})
    if want("sqr"):
        from paper_2604_21566_gb300 import workloads as W
        rows = []
        for m in (32, 128, 256):
            x, _, _ = W.batched_mul(m)
            a = _dv(x)
            p = torch.empty((x.shape[0], 2 * m), dtype=torch.int32, device="cuda")
            t_mul, _ = timer.ms(lambda: dot.mul(a, a, p, ctx=ctx), 10)
            t_sqr, _ = timer.ms(lambda: dot.sqr(a, p, ctx=ctx), 10)
            sel = np.random.default_rng(m).integers(0, x.shape[0], 512)
            ok = np.array_equal(_hs(p)[sel], oracle.sqr(x[sel]))
            rows.append({"m_limbs": m, "ops": x.shape[0], "ms_mul": round(t_mul, 4), "ms_sqr": round(t_sqr, 4),
                         "speedup_sqr_vs_mul": round(t_mul / t_sqr, 3), "bit_exact_sample": bool(ok)})
        emit("batched_square", {"workload": "2^16 operands at 1024/4096/8192 bits", "sizes": rows})
    if want("kara"):
        rows = []
        for m, batch in ((1024, 4096), (2048, 2048), (4096, 1024), (8192, 256)):
            g = np.random.default_rng(5000 + m)
            x = g.integers(0, 2 ** 32, (batch, m), dtype=np.uint64).astype(np.uint32)
            y = g.integers(0, 2 ** 32, (batch, m), dtype=np.uint64).astype(np.uint32)
            a, b = _dv(x), _dv(y)
            p = torch.empty((batch, 2 * m), dtype=torch.int32, device="cuda")
            ms, _ = timer.ms(lambda: dot.mul_karatsuba(a, b, p, ctx=ctx), 5)
            sel = np.arange(0, batch, max(1, batch // 4))
            ok = np.array_equal(_hs(p)[sel], oracle.mul(x[sel], y[sel], threads=8))
            rows.append({"m_limbs": m, "bits": 32 * m, "ops": batch, "ms": round(ms, 4),
                         "schoolbook_equiv_tera_products_s": round(batch * m * m / (ms * 1e-3) / 1e12, 3),
                         "bit_exact_sample": bool(ok)})
        emit("karatsuba", {"workload": "Karatsuba above 512 limbs: 32k..262k-bit products",
                           "note": "schoolbook-equivalent rate = batch m^2 / time", "sizes": rows})
    assert ctx.check() == dot.OK
    ctx.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--suite", action="store_true",
                    help="measure every workload row (one JSON line each) instead of the bench step")
    ap.add_argument("--profile-case", action="store_true",
                    help="run only the small ncu case of the dominant kernel")
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--only", default="", help="--suite rows to run: mix,mul,mixed,shared,splitk,unsat,mulx,sqr,kara")
    ap.add_argument("--case", choices=["add", "long", "mul", "shared", "shared2p18", "shared128", "mixed"],
                    default="add",
                    help="which kernel --profile-case runs")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["dot", "reference"], default="dot")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-rows", action="store_true",
                    help="skip the correctness-mix, multiply, mixed-batch and shared-operand rows")
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
