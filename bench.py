#!/usr/bin/env python
"""Benchmark of the exact sparse polynomial product on GB300.

One step = one pm_polymul call (pack + partition + range kernel + compaction)
on the dense four-variable workload: f and g each hold all 10,626 monomials
of total degree <= 20 with seeded coefficients mod 2^61-1 (112,911,876 term
products collapsing to 135,751 result terms).  Inputs are resident in HBM;
L2 is flushed (256 MiB write) between timed steps, outside the step's events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica of the product on its
own GPU (independent products, no collective on the data path); value is the
total term products of all ranks divided by the slowest rank's time.

Rank 0 prints one JSON line.  ``--impl reference`` times the CPU oracle (the
plain schoolbook product of oracle/oracle.c) on a bounded sample of the same
workload on the host cores.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact term products/sec (1 GB300, % roofline); batched vs plain speedup; p99 ms"
UNIT = "term products/s"
WORKLOAD = ("dense 4-variable product: f, g = all 10,626 monomials of total degree <= 20, "
            "coefficients mod 2^61-1, 16-bit fields (112,911,876 term products -> 135,751 terms)")
FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return
    import oracle
    import polygen
    w = polygen.workload_c2()
    rows = 1000                                   # bounded sample: 1000 rows of f x all of g
    fe, fc = w.f.exps[:rows], w.f.coefs[:rows]
    prods = rows * w.g.n
    for _ in range(args.warmup):
        oracle.mul(w.nvars, w.field_bits, "m61", fe, fc, w.g.exps, w.g.coefs)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.mul(w.nvars, w.field_bits, "m61", fe, fc, w.g.exps, w.g.coefs)
        times.append(time.perf_counter() - t0)
    sec = statistics.mean(times)
    value = prods / sec
    sample = f"first {rows} terms of f x all {w.g.n} terms of g ({prods} term products) per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64 mod 2^61-1", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="pm_clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                    rows.append((ts + frac, parts))
                except ValueError:
                    continue
        os.unlink(self.path)
        inside = [p for ts, p in rows if t0 - 0.1 <= ts <= t1 + 0.1] or [p for _, p in rows]
        sm = [float(p[2]) for p in inside if p[2].replace(".", "").isdigit()]
        smax = [float(p[3]) for p in inside if p[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in inside for i in range(4) if p[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(inside)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def _dev(torch, np, poly, kind="m61"):
    e = torch.from_numpy(poly.exps.view(np.int32).copy()).cuda()
    c = torch.from_numpy(poly.coefs.view(np.int64).copy()).cuda()
    return e, c


def time_product(P, torch, w, steps, warmup, flush, kind="m61", stream=None):
    """Device time of `steps` pm_polymul calls on resident inputs."""
    import numpy as np
    f = _dev(torch, np, w.f)
    g = _dev(torch, np, w.g)
    cap = P.out_bound(w.field_bits, f[0], g[0])
    words = 1 if kind == "m61" else 2
    out = (torch.empty(cap, dtype=torch.int64, device="cuda"),
           torch.empty((cap, 2) if words == 2 else (cap,), dtype=torch.int64, device="cuda"))
    for _ in range(warmup):
        P.polymul(w.field_bits, f[0], f[1], g[0], g[1], kind=kind, out=out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stats = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record()
        r = P.polymul(w.field_bits, f[0], f[1], g[0], g[1], kind=kind, out=out)
        ev[k][1].record()
        stats.append(r.stats)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return ms, stats, r


def probe_peak(P, torch):
    """Measured rate of the per-term-product arithmetic (register-only)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 1 << 14
    sink = torch.empty(blocks * threads, dtype=torch.int64, device="cuda")
    for _ in range(2):
        P.probe_mac(blocks, threads, iters, sink)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        P.probe_mac(blocks, threads, iters, sink)
        b.record()
        torch.cuda.synchronize()
        best = max(best, blocks * threads * 4 * iters / (a.elapsed_time(b) * 1e-3))
    return best


def traffic_for(kernel: str, workload_key: str):
    """dram bytes per launch from the committed ncu summary, or None if the
    kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = d.get(workload_key)
    if not ent or ent.get("kernel") != kernel:
        return None
    src = os.path.join(ROOT, "paper_1303_7425_gb300", "csrc", ent.get("source", "pm_range.cu"))
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return ent.get("dram_bytes_per_launch") if h == ent.get("source_sha256_16") else None


def e2e_product(P, torch, w, steps, warmup):
    """The same product through the public API from pinned host buffers:
    host->device copy of the inputs, the call, device->host copy of the
    result, all inside the timed region."""
    import numpy as np
    hf = [torch.from_numpy(w.f.exps.view(np.int32).copy()).pin_memory(),
          torch.from_numpy(w.f.coefs.view(np.int64).copy()).pin_memory()]
    hg = [torch.from_numpy(w.g.exps.view(np.int32).copy()).pin_memory(),
          torch.from_numpy(w.g.coefs.view(np.int64).copy()).pin_memory()]
    df = [torch.empty_like(x, device="cuda") for x in hf]
    dg = [torch.empty_like(x, device="cuda") for x in hg]
    cap = None
    hk = hc = None
    times = []
    h2d = sum(x.numel() * x.element_size() for x in hf + hg)
    d2h = 0
    for k in range(warmup + steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for s_, d_ in zip(hf + hg, df + dg):
            d_.copy_(s_, non_blocking=True)
        r = P.polymul(w.field_bits, df[0], df[1], dg[0], dg[1])
        if hk is None or hk.shape[0] < r.n:
            hk = torch.empty(r.n, dtype=torch.int64).pin_memory()
            hc = torch.empty(r.n, dtype=torch.int64).pin_memory()
        hk[:r.n].copy_(r.keys, non_blocking=True)
        hc[:r.n].copy_(r.coefs, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        d2h = r.n * 16
        if k >= warmup:
            times.append(a.elapsed_time(b))
    return times, h2d, d2h


def cpu_baseline(w):
    import oracle
    t0 = time.perf_counter()
    he, hc = oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    dt = time.perf_counter() - t0
    return {"value": w.term_products / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the full workload once ({w.term_products} term products, {dt:.1f} s, single thread)",
            "n_out": int(len(he))}


def cpu_alg1(w, rows=2000):
    import oracle
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.mul_alg1(w.nvars, w.field_bits, "m61", w.f.exps[:rows], w.f.coefs[:rows], w.g.exps, w.g.coefs,
                    l=64, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": rows * w.g.n / dt, "unit": UNIT, "cores": threads, "kind": "paper Alg. 1 on CPU threads",
            "sample": f"first {rows} terms of f x all of g"}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1303_7425_gb300 as P
    import polygen

    rank, local, world = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P.lib()  # fails loudly if the CUDA library is missing

    w = polygen.workload_c2()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    products = w.term_products

    # warm-up (also fills the stream-ordered allocator's pool)
    time_product(P, torch, w, 1, args.warmup, flush)
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    t0 = time.time()
    ms, stats, r = time_product(P, torch, w, args.steps, 0, flush)
    torch.cuda.synchronize()
    t1 = time.time()
    if dist:
        dist.barrier()
    clocks = sampler.stop(t0, t1)

    ms_step = statistics.mean(ms)
    if dist:
        tt = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_step = float(tt.item())
    value = world * products / (ms_step * 1e-3)
    kern_ms = statistics.mean(s["ms_range_kernel"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)

    out = None
    if rank == 0:
        peak = probe_peak(P, torch)
        achieved = products / (kern_ms * 1e-3)
        kname = "k_range_direct<M61>" if stats[-1]["strategy"] == "direct" else "k_range_sort<M61>"
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": UNIT, "frac": achieved / peak,
                "traffic": traffic_for(kname, "c2_m61"), "kernel": kname,
                "kernel_ms": kern_ms, "kernel_share_of_step": kern_ms / ms_step,
                "peak_source": "measured on this GPU in this run: register-only M61 multiply-accumulate probe "
                               "(key add + 61x61 product + Mersenne fold + modular add per term product)"}
        e2e_ms, h2d, d2h = e2e_product(P, torch, w, max(5, min(args.steps, 50)), 3)
        e2e_val = products / (statistics.mean(e2e_ms) * 1e-3)
        extras = {}
        if not args.no_extras:
            wi = polygen.workload_c2("i64")
            ms_i, st_i, _ = time_product(P, torch, wi, 20, 3, flush, kind="i64")
            extras["c2_int64_acc128"] = {"value": wi.term_products / (statistics.mean(ms_i) * 1e-3), "unit": UNIT,
                                         "ms_per_step": statistics.mean(ms_i),
                                         "kernel_ms": statistics.mean(s["ms_range_kernel"] for s in st_i)}
            w3 = polygen.workload_c3()
            ms_3, st_3, r3 = time_product(P, torch, w3, 5, 2, flush)
            extras["c3_sparse5v_50000x50000"] = {
                "value": w3.term_products / (statistics.mean(ms_3) * 1e-3), "unit": UNIT,
                "ms_per_step": statistics.mean(ms_3), "n_out": r3.n,
                "kernel_ms": statistics.mean(s["ms_range_kernel"] for s in st_3),
                "kernel_frac_of_probe": w3.term_products / (statistics.mean(s["ms_range_kernel"] for s in st_3) * 1e-3) / peak}
        cpu = None if (args.no_cpu or world > 1) else cpu_baseline(w)
        if cpu is not None:
            extras["cpu_alg1_threads"] = cpu_alg1(w)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64 mod 2^61-1", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "strategy": stats[-1]["strategy"], "ranges": stats[-1]["n_ranges"],
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "roofline": roof,
            "cpu_baseline": {k: v for k, v in cpu.items() if k != "n_out"} if cpu else None,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "n_out": r.n,
            "host_syncs_per_step": stats[-1]["host_syncs"],
            "extras": extras,
        }
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
