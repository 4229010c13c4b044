#!/usr/bin/env python
"""Benchmark of the exact sparse polynomial product on GB300.

One step = one whole product h = f * g (pack + partition + FindEdge + range
kernel + compaction), replayed as one captured CUDA graph (pm_plan_run) on
the largest single-GPU workload: the sparse five-variable product, f and g
each 50,000 distinct terms of the box with degree caps (6, 8, 10, 12, 16),
coefficients mod 2^61-1 (2.5e9 term products collapsing to 3,824,065 result
terms).  Inputs are resident in HBM; L2 is flushed (256 MiB write) between
timed steps, outside the step's events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload sparse5v|dense4v|sparse4v|batch]

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
WORKLOADS = {
    "sparse5v": ("sparse 5-variable product: f, g = 50,000 distinct terms each of the box with degree caps "
                 "(6,8,10,12,16), coefficients mod 2^61-1, 12-bit fields (2.5e9 term products -> 3,824,065 terms)"),
    "dense4v": ("dense 4-variable product: f, g = all 10,626 monomials of total degree <= 20, "
                "coefficients mod 2^61-1, 16-bit fields (112,911,876 term products -> 135,751 terms)"),
    "sparse4v": ("sparse 4-variable product: f, g = 1000 distinct terms each of total degree <= 12, "
                 "coefficients mod 2^61-1, 16-bit fields (1e6 term products)"),
}
# the oracle's bounded samples: rows of f times all of g
CPU_ROWS = {"sparse5v": 1000, "dense4v": 10626, "sparse4v": 1000}
REF_ROWS = {"sparse5v": 200, "dense4v": 1000, "sparse4v": 1000}
FLUSH_BYTES = 256 << 20
# Sec. 8(d)'s algorithmic operation count of one term product in the split
# multiply form: four 32 x 32 -> 64 multiplies; about fourteen simple ops
# (key add, guard test, the adds of the partial products, the Mersenne fold,
# one modular add)
OPS_WIDE, OPS_SIMPLE = 4, 14
ISSUE_LANES_PER_CLK = 128     # 4 schedulers per SM, one 32-lane warp instruction each per clock


def _workload(name):
    import polygen
    return {"sparse5v": polygen.workload_sparse5v, "dense4v": polygen.workload_dense4v,
            "sparse4v": polygen.workload_sparse4v}[name]()


def hbm_peak():
    """(GB/s, source) -- the measured copy bandwidth of the GB300s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    ap.add_argument("--example-power", type=int, default=None,
                    help="with --workload paper_ex2|paper_ex3: a smaller exponent than the paper's (profiling)")
    ap.add_argument("--shard", action="store_true",
                    help="one product split over the ranks by output key range (Alg. 2) instead of replicas")
    ap.add_argument("--workload", default="sparse5v", choices=["sparse5v", "dense4v", "sparse4v", "batch", "paper_ex2", "paper_ex3"],
                    help="what the timed steps run; the line reports that workload (default: the largest)")
    ap.add_argument("--batch-count", type=int, default=4096, help="products of the batched workload")
    ap.add_argument("--serving-count", type=int, default=3000, help="requests of the serving workload")
    return ap.parse_args()


def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest x over all ranks (every rank gets it); x itself without
    a process group.  device: where the backend reduces ("cuda" for NCCL,
    "cpu" for gloo)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: int, world: int, slowest_ms: float) -> float:
    """Units per second of the whole job: every rank processes its own
    units (replicas, weak scaling), and the job takes as long as the
    slowest rank."""
    return world * units_per_rank / (slowest_ms * 1e-3)


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
    name = args.workload if args.workload in WORKLOADS else "sparse5v"
    w = _workload(name)
    rows = min(REF_ROWS[name], w.f.n)             # bounded sample: rows of f x all of g
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
        "config": {"workload": WORKLOADS[name], "sample": sample},
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
    """Measured rate of the per-term-product arithmetic loop (register-only,
    pm_probe_mac; it also carries one operand-advance add and mask)."""
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


def oprate_peak(P, torch):
    """The integer-op bound of one term product, from instruction rates
    measured on this GPU (register-only probes, pm_probe_oprate) and the
    pipes they run on.  On GB300 the simple ops (three-input add and logic
    op, funnel shift) issue to the ALU pipe and the multiplies to the
    FMA-heavy pipe, each about 64 lanes per SM per clock; a 32 x 32 -> 64
    multiply keeps the FMA-heavy pipe twice as long as a 32-bit one; an SM
    issues at most 128 lane-instructions per clock.  A term product needs
    OPS_WIDE wide multiplies and OPS_SIMPLE simple ops, so an SM needs at
    least max(OPS_WIDE / r_wide, OPS_SIMPLE / r_simple,
    (OPS_WIDE + OPS_SIMPLE) / 128) clocks per product, with r_wide the
    larger of the measured wide rate and half the 32-bit multiply rate."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads = sms * 4, 256
    sink = torch.empty(blocks * threads, dtype=torch.int64, device="cuda")
    clk = torch.zeros(2, dtype=torch.int64, device="cuda")
    rates, mhz = {}, []
    for op in ("imad_wide", "imad", "imad_hi", "iadd3", "lop3", "shf"):
        iters = 1 << 16
        P.probe_oprate(op, blocks, threads, iters >> 4, sink, clk)      # warm-up
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            per_step = P.probe_oprate(op, blocks, threads, iters, sink, clk)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            cyc, ns = (int(x) for x in clk.cpu().tolist())
            f_ghz = cyc / ns if ns > 0 else float("nan")
            ops = blocks * threads * iters * per_step
            per_sm_clk = ops / (ms * 1e-3) / (sms * f_ghz * 1e9)
            if best is None or per_sm_clk > best[0]:
                best = (per_sm_clk, ops / (ms * 1e-3), f_ghz * 1e3)
        rates[op] = {"per_sm_per_clk": best[0], "lane_ops_per_s": best[1], "sm_mhz": best[2]}
        mhz.append(best[2])
    r_simple = max(rates[k]["per_sm_per_clk"] for k in ("iadd3", "lop3", "shf"))
    r_wide = max(rates["imad_wide"]["per_sm_per_clk"], rates["imad"]["per_sm_per_clk"] / 2)
    clk_per_product = max(OPS_WIDE / r_wide, OPS_SIMPLE / r_simple, (OPS_WIDE + OPS_SIMPLE) / ISSUE_LANES_PER_CLK)
    f_mhz = statistics.median(mhz)
    peak = sms * f_mhz * 1e6 / clk_per_product
    return {"peak": peak, "clk_per_product_per_sm": clk_per_product, "r_wide": r_wide, "r_simple": r_simple,
            "sm_mhz": f_mhz, "sms": sms, "ops_per_product": {"wide_multiply": OPS_WIDE, "simple": OPS_SIMPLE},
            "rates": {k: round(v["per_sm_per_clk"], 2) for k, v in rates.items()}}


def kernel_source_hash(source: str, region=None):
    """sha256 (16 hex digits) of a kernel's source text: the whole file, or
    the text from the line starting with region[0] up to (not including) the
    line starting with region[1]."""
    path = os.path.join(ROOT, "paper_1303_7425_gb300", "csrc", source)
    try:
        text = open(path, encoding="utf-8").read()
    except OSError:
        return None
    if region:
        a = text.find("\n" + region[0])
        b = text.find("\n" + region[1], a + 1)
        if a < 0 or b < 0:
            return None
        text = text[a + 1:b + 1]
    return hashlib.sha256(text.encode("utf-8")).hexdigest()[:16]


def traffic_for(kernel: str, workload_key: str):
    """dram bytes per launch from the committed ncu summary, or None if the
    kernel's source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = d.get(workload_key)
    if not ent or ent.get("kernel") != kernel:
        return None
    h = kernel_source_hash(ent.get("source", "pm_direct.cu"), ent.get("region"))
    return ent.get("dram_bytes_per_launch") if h and h == ent.get("source_sha256_16") else None


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


def time_plan(P, torch, w, steps, warmup, flush, kind="m61"):
    """Device time of `steps` replays of a captured plan (pm_plan_run): every
    kernel of the product re-runs on the resident inputs each step; the
    result size is read (pm_plan_finish) after each step, outside the
    events.  Returns (ms list, result size) or None if not captured."""
    import numpy as np
    f = _dev(torch, np, w.f)
    g = _dev(torch, np, w.g)
    cap = P.out_bound(w.field_bits, f[0], g[0])
    words = 1 if kind == "m61" else 2
    out = (torch.empty(cap, dtype=torch.int64, device="cuda"),
           torch.empty((cap, 2) if words == 2 else (cap,), dtype=torch.int64, device="cuda"))
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out, kind=kind)
    try:
        if not plan.captured:
            return None
        for _ in range(warmup):
            plan.run()
            plan.finish()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        n = 0
        for k in range(steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record()
            plan.run()
            ev[k][1].record()
            n = plan.finish()
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], n
    finally:
        plan.close()


def e2e_plan(P, torch, w, steps, warmup):
    """The plan path end to end: host->device copy of the inputs from pinned
    memory into the plan's input buffers, the replay, the result size, and
    the device->host copy of the result, all inside the timed region."""
    import numpy as np
    hf = [torch.from_numpy(w.f.exps.view(np.int32).copy()).pin_memory(),
          torch.from_numpy(w.f.coefs.view(np.int64).copy()).pin_memory()]
    hg = [torch.from_numpy(w.g.exps.view(np.int32).copy()).pin_memory(),
          torch.from_numpy(w.g.coefs.view(np.int64).copy()).pin_memory()]
    df = [x.cuda() for x in hf]
    dg = [x.cuda() for x in hg]
    cap = P.out_bound(w.field_bits, df[0], dg[0])
    out = (torch.empty(cap, dtype=torch.int64, device="cuda"), torch.empty(cap, dtype=torch.int64, device="cuda"))
    plan = P.Plan(w.field_bits, df[0], df[1], dg[0], dg[1], out)
    hk = torch.empty(cap, dtype=torch.int64).pin_memory()
    hc = torch.empty(cap, dtype=torch.int64).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in hf + hg)
    times, d2h = [], 0
    direct_host = True
    try:
        for k in range(warmup + steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for s_, d_ in zip(hf + hg, df + dg):
                d_.copy_(s_, non_blocking=True)
            plan.run()
            # the result lands in the pinned host buffers on the device side
            # (pm_plan_finish_to_host): one host wait per step; host buffers
            # the device cannot address take the size first, then copies
            if direct_host:
                try:
                    n = plan.finish_to_host(hk, hc)
                except P.PolymulError as e:
                    if e.code != -1:
                        raise
                    direct_host = False
            if not direct_host:
                n = plan.finish()
                hk[:n].copy_(out[0][:n], non_blocking=True)
                hc[:n].copy_(out[1][:n], non_blocking=True)
            b.record()
            torch.cuda.synchronize()
            d2h = n * 16
            if k >= warmup:
                times.append(a.elapsed_time(b))
    finally:
        plan.close()
    return times, h2d, d2h


def _device_product(torch, np, w, cap=None):
    f = (torch.from_numpy(w.f.exps.view(np.int32).copy()).cuda(), torch.from_numpy(w.f.coefs.view(np.int64).copy()).cuda())
    g = (torch.from_numpy(w.g.exps.view(np.int32).copy()).cuda(), torch.from_numpy(w.g.coefs.view(np.int64).copy()).cuda())
    cap = cap if cap is not None else max(w.f.n * w.g.n, 1)
    out = (torch.empty(cap, dtype=torch.int64, device="cuda"), torch.empty(cap, dtype=torch.int64, device="cuda"))
    return dict(field_bits=w.field_bits, kind=w.kind, f_exps=f[0], f_coefs=f[1], g_exps=g[0], g_coefs=g[1], out=out)


def bench_paper_example(P, torch, nm, peak=None, power=None):
    """The paper's Example 2 or 3 (Sec. 6) at full size, mod p, through
    pm_polymul (hashed windows): one warm call, then the mean of two.  At a
    smaller power (a profiling aid) the hashed windows are asked for, since
    the library would pick the direct windows for the smaller box."""
    import numpy as np

    import polygen
    ctx = {"ex2": "Fermi GPU, FP64: 71 s; 64 Xeon cores, integers: 30.2 s (Sec. 6)",
           "ex3": "Fermi GPU, FP64: 129 s; 64 Xeon cores, integers: 29.7 s (Sec. 6)"}
    wx = polygen.paper_example(nm, power)
    fx, gx = _dev(torch, np, wx.f), _dev(torch, np, wx.g)
    capx = ({"ex2": 312855140, "ex3": 144049555}[nm] + 16 if power is None
            else P.out_bound(wx.field_bits, fx[0], gx[0]))
    outx = (torch.empty(capx, dtype=torch.int64, device="cuda"),
            torch.empty(capx, dtype=torch.int64, device="cuda"))
    strat = "auto" if power is None else "hash"
    P.polymul(wx.field_bits, fx[0], fx[1], gx[0], gx[1], out=outx, strategy=strat)
    tx = []
    for _ in range(2):
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record()
        rx = P.polymul(wx.field_bits, fx[0], fx[1], gx[0], gx[1], out=outx, strategy=strat)
        b_.record()
        torch.cuda.synchronize()
        tx.append(a_.elapsed_time(b_))
    value = wx.term_products / (statistics.mean(tx) * 1e-3)
    res = {"value": value, "unit": UNIT, "ms_per_step": statistics.mean(tx), "n_out": rx.n,
           "term_products": wx.term_products, "strategy": rx.stats["strategy"],
           "window_rounds": rx.stats["refine_rounds"], "window_runs": rx.stats["n_ranges"],
           "workload": wx.note, "paper_context": ctx[nm], "frac": value / peak if peak else None}
    del fx, gx, outx
    torch.cuda.empty_cache()
    return res


def bench_batched(P, torch, count, tune=True):
    """The batched workload: `count` independent sparse products -- one captured batched pass
    versus one pm_polymul launch per product, on the same GPU."""
    import numpy as np

    import oracle
    import polygen
    ws = polygen.workload_sparse_batch(count)
    prods = [_device_product(torch, np, w) for w in ws]
    tp = sum(w.term_products for w in ws)
    best = P.batch_autotune(prods)[0] if tune else {}
    plan = P.BatchPlan(prods, **best)
    plan.run()
    res, st = plan.finish()
    times = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    res, st = plan.finish()
    plan.close()
    failed = sum(1 for s_, _ in res if s_ != 0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for pr in prods:
        P.polymul(pr["field_bits"], pr["f_exps"], pr["f_coefs"], pr["g_exps"], pr["g_coefs"], out=pr["out"])
    b.record()
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b)
    # parity of the batched results on sampled products
    plan = P.BatchPlan(prods, **best)
    plan.run()
    res, _ = plan.finish()
    plan.close()
    rng = np.random.default_rng(0)
    small = [k for k, w in enumerate(ws) if w.term_products <= 1_000_000]
    checked = 0
    for k in rng.choice(small, size=min(8, len(small)), replace=False):
        w = ws[k]
        e, c = oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
        n = res[k][1]
        ok = n == len(e) and np.array_equal(prods[k]["out"][1][:n].cpu().numpy().view(np.uint64), c)
        checked += 1 if ok else 0
    ms = statistics.mean(times)
    # the pass's HBM roofline: every input term read once (exponents and
    # coefficient), every result term written once (key and coefficient)
    n_out = sum(n for _, n in res)
    in_bytes = sum((w.f.n + w.g.n) * (4 * w.nvars + 8) for w in ws)
    alg_bytes = in_bytes + 16 * n_out
    peak, peak_src = hbm_peak()
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    del prods
    torch.cuda.empty_cache()
    return {"products": count, "term_products": tp, "batched_ms": ms, "batched_value": tp / (ms * 1e-3),
            "result_terms": n_out,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "algorithmic_bytes": alg_bytes, "peak_source": peak_src,
                         "scope": "the whole batched pass (B1-B4) per graph replay"},
            "plain_ms": plain_ms, "plain_value": tp / (plain_ms * 1e-3), "batched_vs_plain_speedup": plain_ms / ms,
            "unit": UNIT, "options": best, "ranges": st["n_ranges"], "work_items": st["work_items"],
            "graph": bool(st["graph"]), "failed": failed, "oracle_checked": checked,
            "oracle_sampled": int(min(8, len(small)))}


def bench_sparse_large(P, torch, np, polygen, flush):
    """A sparse five-variable product whose result is about as large as its
    4e8 term products (20,000 x 20,000 terms, exponents up to 1023, 12-bit
    fields): the default strategy (bucketed) against the sort strategy on
    the same GPU, results compared on the device."""
    w = polygen.sparse_product(polygen.Stream(polygen.BASE_SEED + 5, 0), 5, 20000, 20000)
    f, g = _dev(torch, np, w.f), _dev(torch, np, w.g)
    cap = min(w.term_products, P.out_bound(w.field_bits, f[0], g[0]))
    outs = [(torch.empty(cap, dtype=torch.int64, device="cuda"), torch.empty(cap, dtype=torch.int64, device="cuda"))
            for _ in range(2)]
    res = {}
    for k, strat in enumerate(("auto", "sort")):
        reps = 3 if strat == "auto" else 1
        P.polymul(w.field_bits, f[0], f[1], g[0], g[1], out=outs[k], strategy=strat)   # warm-up
        ts = []
        for q in range(reps):
            flush.fill_(q)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record()
            r = P.polymul(w.field_bits, f[0], f[1], g[0], g[1], out=outs[k], strategy=strat)
            b_.record()
            torch.cuda.synchronize()
            ts.append(a_.elapsed_time(b_))
        res[strat] = (statistics.mean(ts), r)
    same = (res["auto"][1].n == res["sort"][1].n and torch.equal(outs[0][0][:res["auto"][1].n], outs[1][0][:res["sort"][1].n])
            and torch.equal(outs[0][1][:res["auto"][1].n], outs[1][1][:res["sort"][1].n]))
    ms, r = res["auto"]
    del outs, f, g
    torch.cuda.empty_cache()
    return {"workload": "5 vars, 20,000 x 20,000 distinct terms, exponents uniform in [0, 1023], 12-bit fields, "
                        "mod 2^61-1", "term_products": w.term_products, "n_out": r.n, "strategy": r.stats["strategy"],
            "ms": ms, "value": w.term_products / (ms * 1e-3), "unit": UNIT,
            "kernel_phase_ms": r.stats["ms_range_kernel"], "large_buckets": r.stats["refine_rounds"],
            "sort_strategy_ms": res["sort"][0], "speedup_vs_sort_strategy": res["sort"][0] / ms,
            "same_result_as_sort_strategy": bool(same)}


def bench_serving(P, torch, count, rate_hz, tune=True):
    """Serving: Poisson arrivals at `rate_hz`, 95% batch-distribution and 5%
    dense 4-variable products, continuous batching under a 64 GiB HBM budget."""
    import numpy as np

    import oracle
    import polygen
    from paper_1303_7425_gb300.serving import serve
    reqs = polygen.workload_serving_mix(rate_hz, count)
    prods = [_device_product(torch, np, r.work, cap=(200_000 if r.dense else None)) for r in reqs]
    rep = serve([(r.t_arrival, pr) for r, pr in zip(reqs, prods)], [r.work.term_products for r in reqs],
                server_kwargs=dict(device_budget=64 << 30, streams=4, max_batch=256))
    # every result equals the same product computed alone
    same = 0
    for k, (r, pr) in enumerate(zip(reqs, prods)):
        n = rep["done"][k]["n"]
        if r.dense:
            alone = P.polymul(pr["field_bits"], pr["f_exps"], pr["f_coefs"], pr["g_exps"], pr["g_coefs"])
            ok = alone.n == n and torch.equal(alone.coefs, pr["out"][1][:n]) and torch.equal(alone.keys, pr["out"][0][:n])
        else:
            cap = max(r.work.f.n * r.work.g.n, 1)
            out = (torch.empty(cap, dtype=torch.int64, device="cuda"), torch.empty(cap, dtype=torch.int64, device="cuda"))
            alone = P.polymul(pr["field_bits"], pr["f_exps"], pr["f_coefs"], pr["g_exps"], pr["g_coefs"], out=out)
            ok = alone.n == n and torch.equal(alone.coefs, pr["out"][1][:n]) and torch.equal(alone.keys, pr["out"][0][:n])
        same += 1 if ok else 0
    rng = np.random.default_rng(1)
    small = [k for k, r in enumerate(reqs) if not r.dense and r.work.term_products <= 500_000]
    checked = 0
    for k in rng.choice(small, size=min(8, len(small)), replace=False):
        w = reqs[k].work
        e, c = oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
        n = rep["done"][k]["n"]
        checked += 1 if (n == len(e) and np.array_equal(prods[k]["out"][1][:n].cpu().numpy().view(np.uint64), c)) else 0
    del prods
    torch.cuda.empty_cache()
    return {"requests": count, "rate_hz": rate_hz, "dense_requests": int(sum(r.dense for r in reqs)),
            "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"], "mean_ms": rep["mean_ms"],
            "value": rep["term_products_per_s"], "unit": UNIT, "failed": rep["failed"],
            "same_alone_and_in_mix": same, "oracle_checked": checked, "oracle_sampled": int(min(8, len(small))),
            "batches": rep["state"]["batches"], "max_batches_in_flight": rep["state"]["max_in_flight"],
            "hbm_budget_gib": 64}


def cpu_baseline(w, rows):
    """The oracle (single thread, as it stands) on a bounded sample: the
    first `rows` terms of f times all of g."""
    import oracle
    rows = min(rows, w.f.n)
    t0 = time.perf_counter()
    oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps[:rows], w.f.coefs[:rows], w.g.exps, w.g.coefs)
    dt = time.perf_counter() - t0
    return {"value": rows * w.g.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {rows} terms of f x all {w.g.n} terms of g ({rows * w.g.n} term products, "
                      f"{dt:.1f} s, single thread)"}


def cpu_alg1(w, rows):
    import oracle
    threads = os.cpu_count() or 1
    rows = min(rows, w.f.n)
    t0 = time.perf_counter()
    oracle.mul_alg1(w.nvars, w.field_bits, "m61", w.f.exps[:rows], w.f.coefs[:rows], w.g.exps, w.g.coefs,
                    l=64, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": rows * w.g.n / dt, "unit": UNIT, "cores": threads, "kind": "paper Alg. 1 on CPU threads",
            "sample": f"first {rows} terms of f x all of g ({dt:.1f} s)"}


def kernel_roofline(products, kern_ms, step_ms, kname, traffic_key, op, probe, range_step_ms):
    achieved = products / (kern_ms * 1e-3)
    return {"bound": "alu", "achieved": achieved, "peak": op["peak"], "unit": UNIT, "frac": achieved / op["peak"],
            "traffic": traffic_for(kname, traffic_key), "kernel": kname,
            "kernel_ms": kern_ms, "range_step_ms": range_step_ms, "kernel_share_of_step": kern_ms / step_ms,
            "peak_source": ("derived from instruction rates measured on this GPU in this run (register-only "
                            "probes): %d wide multiplies + %d simple ops per term product; wide multiplies at "
                            "%.1f, simple ops at %.1f lane-ops per SM per clock (FMA-heavy and ALU pipes), issue "
                            "limit 128; %.3f clocks per product per SM, %d SMs at %.0f MHz"
                            % (OPS_WIDE, OPS_SIMPLE, op["r_wide"], op["r_simple"], op["clk_per_product_per_sm"],
                               op["sms"], op["sm_mhz"])),
            "frac_of_mac_probe": achieved / probe, "mac_probe": probe}


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

    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    if args.workload == "batch":  # profiling aid: the batched pass as the timed step
        print(json.dumps(bench_batched(P, torch, args.batch_count, tune=not args.no_tune)))
        return
    if args.workload in ("paper_ex2", "paper_ex3"):  # profiling aid: the paper's Example 2 or 3
        print(json.dumps(bench_paper_example(P, torch, args.workload[6:], power=args.example_power)))
        return
    name = args.workload
    w = _workload(name)
    products = w.term_products
    tuned = None
    if not args.no_tune:
        f = _dev(torch, np, w.f)
        g = _dev(torch, np, w.g)
        tuned = P.autotune(w.field_bits, f[0], f[1], g[0], g[1])[0]
        del f, g

    # warm-up (also fills the stream-ordered allocator's pool)
    time_product(P, torch, w, 1, args.warmup, flush)
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    t0 = time.time()
    # the same product as a captured plan: one CUDA graph per step, every
    # kernel re-run on the resident inputs, no host synchronisation inside
    planned = time_plan(P, torch, w, args.steps, args.warmup, flush)
    # plain calls: the accumulate kernel timed alone with events on its stream
    ms_plain, stats, r = time_product(P, torch, w, max(3, min(args.steps, 10)), 0, flush)
    torch.cuda.synchronize()
    t1 = time.time()
    if dist:
        dist.barrier()
    clocks = sampler.stop(t0, t1)

    ms = planned[0] if planned else ms_plain
    ms_step = max_over_ranks(statistics.mean(ms), dist, "cuda")
    value = whole_job_value(products, world, ms_step)
    kern_ms = statistics.mean(s["ms_range_kernel"] for s in stats)
    # kernels per timed step: the call's launches (+ the plan's two check kernels)
    launches = args.steps * (stats[-1]["kernel_launches"] + (2 if planned else 0))

    out = None
    if rank == 0:
        op = oprate_peak(P, torch)
        probe = probe_peak(P, torch)
        kname = {"direct": "k_direct", "sort": "k_range_sort", "hash": "k_hash"}[stats[-1]["strategy"]]
        roof = kernel_roofline(products, kern_ms, ms_step, kname, name, op, probe,
                               statistics.mean(s["ms_range_step"] for s in stats))
        if planned:
            e2e_ms, h2d, d2h = e2e_plan(P, torch, w, max(5, min(args.steps, 30)), 3)
        else:
            e2e_ms, h2d, d2h = e2e_product(P, torch, w, max(5, min(args.steps, 30)), 3)
        e2e_val = products / (statistics.mean(e2e_ms) * 1e-3)
        extras = {f"{name}_plain_call": {"value": products / (statistics.mean(ms_plain) * 1e-3), "unit": UNIT,
                                         "ms_per_step": statistics.mean(ms_plain),
                                         "host_syncs_per_step": stats[-1]["host_syncs"],
                                         "api": "pm_polymul (host reads sizes between steps)"}}
        # the secondary workloads run on one GPU only (with N ranks the
        # others would wait for rank 0 at the closing barrier)
        if not args.no_extras and world == 1:
            try:
                secondary_workloads(extras, P, torch, np, polygen, args, name, flush, op, probe, ms_step)
            except Exception as e:  # the headline line still prints; the failure is reported in it
                extras["secondary_error"] = f"{type(e).__name__}: {e}"
        cpu = None
        if not args.no_cpu and world == 1:
            cpu = cpu_baseline(w, CPU_ROWS[name])
            extras["cpu_alg1_threads"] = cpu_alg1(w, 5 * CPU_ROWS[name])
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64 mod 2^61-1", "data": "synthetic",
            "config": {"workload": WORKLOADS[name], "term_products": products,
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "api": ("pm_plan_run: the whole device path as one CUDA graph, every kernel re-run "
                               "on the resident inputs each step" if planned else "pm_polymul"),
                       "strategy": stats[-1]["strategy"], "ranges": stats[-1]["n_ranges"], "tuned": tuned,
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "n_out": r.n,
            "host_syncs_per_step": 1 if planned else stats[-1]["host_syncs"],
            "oprate": op,
            "extras": extras,
        }
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def secondary_workloads(extras, P, torch, np, polygen, args, name, flush, op, probe, ms_head):
    """The other workloads on this GPU: each config that is not the headline
    (plan replay and accumulate kernel with their own roofline fractions),
    the int64 dense product, the paper's Examples 1-3, the batched pass and
    the serving loop.  Fills `extras` as it goes."""
    for other in ("dense4v", "sparse4v", "sparse5v"):
        if other == name:
            continue
        wo = _workload(other)
        if not args.no_tune:
            fo, go = _dev(torch, np, wo.f), _dev(torch, np, wo.g)
            P.autotune(wo.field_bits, fo[0], fo[1], go[0], go[1])
            del fo, go
        pl = time_plan(P, torch, wo, 20, 3, flush)
        msp, sto, ro = time_product(P, torch, wo, 10, 3, flush)
        step = statistics.mean(pl[0]) if pl else statistics.mean(msp)
        kname = {"direct": "k_direct", "sort": "k_range_sort", "hash": "k_hash"}[sto[-1]["strategy"]]
        km = statistics.mean(s["ms_range_kernel"] for s in sto)
        extras[other] = {"workload": WORKLOADS[other], "value": wo.term_products / (step * 1e-3), "unit": UNIT,
                         "ms_per_step": step, "api": "plan replay" if pl else "pm_polymul",
                         "plain_call_ms": statistics.mean(msp), "n_out": ro.n, "strategy": sto[-1]["strategy"],
                         "kernel": kname, "kernel_ms": km,
                         "kernel_frac": wo.term_products / (km * 1e-3) / op["peak"],
                         "kernel_frac_of_mac_probe": wo.term_products / (km * 1e-3) / probe,
                         "traffic": traffic_for(kname, other)}
    wi = polygen.workload_dense4v("i64")
    ms_i, st_i, _ = time_product(P, torch, wi, 20, 3, flush, kind="i64")
    extras["dense4v_int64_acc128"] = {"value": wi.term_products / (statistics.mean(ms_i) * 1e-3), "unit": UNIT,
                                      "ms_per_step": statistics.mean(ms_i),
                                      "kernel_ms": statistics.mean(s["ms_range_kernel"] for s in st_i)}
    # the paper's Example 1 at full size (Sec. 6): 1.84e10 term products
    we = polygen.paper_example1()
    pe = time_plan(P, torch, we, 5, 2, flush)
    if pe:
        extras["paper_example1"] = {
            "value": we.term_products / (statistics.mean(pe[0]) * 1e-3), "unit": UNIT,
            "ms_per_step": statistics.mean(pe[0]), "n_out": pe[1], "term_products": we.term_products,
            "workload": "f1 = (1+x+y+z+t)^40 times f1 + 1, mod 2^61-1 (plan replay)",
            "frac": we.term_products / (statistics.mean(pe[0]) * 1e-3) / op["peak"],
            "paper_context": "Fermi GPU, FP64 coefficients: 32 s; 64 Xeon cores, integers: 16.1 s (Sec. 6)"}
    # Examples 2 and 3 (hashed windows)
    for nm in ("ex2", "ex3"):
        extras["paper_" + nm] = bench_paper_example(P, torch, nm, op["peak"])
    extras["sparse5v_20000x20000"] = bench_sparse_large(P, torch, np, polygen, flush)
    sb = bench_batched(P, torch, args.batch_count, tune=not args.no_tune)
    extras["sparse_batch_4096"] = sb
    # serving at ~70% of the measured capacity for the request mix: 95%
    # sparse requests at the batched pass's time per product, 5% dense ones
    # at the dense step's time
    ms_dense = extras["dense4v"]["ms_per_step"] if "dense4v" in extras else ms_head
    t_req = 0.95 * sb["batched_ms"] * 1e-3 / args.batch_count + 0.05 * ms_dense * 1e-3
    rate = 0.7 / t_req
    extras["serving_mix"] = bench_serving(P, torch, args.serving_count, rate, tune=not args.no_tune)


def run_sharded(args):
    """One product over all ranks (Alg. 2, Sec. 3): every rank computes the
    same split of the output key space, multiplies its slice and the slices
    are gathered in rank order (paper_1303_7425_gb300.shard.sharded_polymul).
    The whole job makes the product once per step, so the scaling is strong;
    value = the product's term products / the slowest rank's step time."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1303_7425_gb300 as P
    from paper_1303_7425_gb300.shard import sharded_polymul
    rank, local, world = env_rank()
    # a one-rank group when started without torchrun
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", "29531")
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", rank=rank, world_size=world, device_id=torch.device("cuda", local))
    P.lib()  # fails loudly if the CUDA library is missing
    name = args.workload if args.workload in WORKLOADS else "sparse5v"
    w = _workload(name)
    f, g = _dev(torch, np, w.f), _dev(torch, np, w.g)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    run = lambda: sharded_polymul(w.field_bits, f[0], f[1], g[0], g[1])
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    t0 = time.time()
    ts = []
    for k in range(args.steps):
        flush.fill_(k & 255)
        dist.barrier()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        hk, hc, n, st = run()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    t1 = time.time()
    clocks = sampler.stop(t0, t1)
    ms_step = max_over_ranks(statistics.mean(ts), dist, "cuda")
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": w.term_products / (ms_step * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u64 mod 2^61-1", "data": "synthetic",
            "config": {"workload": WORKLOADS[name], "term_products": w.term_products,
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "api": "shard.sharded_polymul: pm_shard_bounds, pm_polymul_range on each rank, "
                              "then the ordered all-gather of the slices",
                       "parallelism": f"key-range shards x{world}"},
            "roofline": None, "cpu_baseline": None, "e2e": None,
            "gpu_launches": args.steps * st["kernel_launches"],
            "gpu_launches_note": "the slice's pm_polymul_range kernels per step; the split's are not counted",
            "clocks": clocks, "n_out": n,
            "slice": {"products": st["slice_products"], "terms": st["slice_terms"]}}))
    dist.barrier()
    dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.shard:
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
