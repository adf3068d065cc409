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
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2604_21566_gb300", "csrc", f)
                  for f in ("dot_addsub.cu", "dot_internal.cuh", "dot_plan.h")]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()

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
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())

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
        value = world * ops_step / (ms_step * 1e-3) / 1e9
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
            "e2e": {"value": round(world * ops_step / (e2e_ms * 1e-3) / 1e9, 4), "unit": "Gop/s",
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
    """Small case for ncu: dot_add on 2^18 pairs of 4096-bit operands
    (403 MB of algorithmic traffic, larger than L2), a few launches."""
    import torch
    from paper_2604_21566_gb300 import dot
    from paper_2604_21566_gb300 import workloads as W
    torch.cuda.set_device(0)
    d = W.addsub_bandwidth(short_batch=1 << 18, long_batch=0)
    x, y = d["add_short"]
    a = torch.from_numpy(x.view(np.int32)).cuda()
    b = torch.from_numpy(y.view(np.int32)).cuda()
    s = torch.empty_like(a)
    c = torch.empty(a.shape[0], dtype=torch.int32, device="cuda")
    ctx = dot.Context(0)
    for _ in range(args.launches):
        dot.add(a, b, out=s, carry=c, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.check() == dot.OK
    print("profile case done")


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--profile-case", action="store_true",
                    help="run only the small ncu case of the dominant kernel")
    ap.add_argument("--launches", type=int, default=3)
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
    if args.profile_case:
        from paper_2604_21566_gb300 import build as B
        B.build()
        profile_case(args)
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
