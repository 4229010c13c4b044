"""Drive the native serving engine with timed arrivals.

``serve(requests, ...)`` submits each request when its arrival time (seconds
from the start) has passed, polls the engine for completions, and reports
per-request latency (completion seen by the engine minus submission), p50 /
p99 and throughput.  The request loop, admission, batching and stream
management are the engine's (pm_server_* in the C library); this module only
replays the arrival schedule.
"""

from __future__ import annotations

import time
from typing import Dict, List, Sequence, Tuple

from ._native import Server


def percentile(xs: Sequence[float], q: float) -> float:
    s = sorted(xs)
    if not s:
        return float("nan")
    k = min(len(s) - 1, max(0, int(round(q / 100.0 * (len(s) - 1)))))
    return s[k]


def serve(requests: List[Tuple[float, dict]], term_products: Sequence[int], server_kwargs=None,
          timeout_s: float = 600.0) -> Dict:
    """requests: (arrival seconds, product dict) sorted by arrival; product
    dicts as for BatchPlan.  term_products[k]: n_f * n_g of request k."""
    srv = Server(**(server_kwargs or {}))
    done: Dict[int, dict] = {}
    try:
        k = 0
        t0 = time.perf_counter()
        n = len(requests)
        while len(done) < n:
            now = time.perf_counter() - t0
            while k < n and requests[k][0] <= now:
                srv.submit(requests[k][1], k)
                k += 1
            for d in srv.progress():
                done[d["tag"]] = d
            if now > timeout_s:
                raise TimeoutError(f"serving did not finish within {timeout_s} s")
        state = srv.state()
    finally:
        srv.close()
    lat = [done[k]["t_done"] - done[k]["t_submit"] for k in range(len(requests))]
    t_first = min(d["t_submit"] for d in done.values())
    t_last = max(d["t_done"] for d in done.values())
    ok = [k for k in range(len(requests)) if done[k]["status"] == 0]
    return {
        "done": done,
        "p50_ms": 1e3 * percentile(lat, 50),
        "p99_ms": 1e3 * percentile(lat, 99),
        "mean_ms": 1e3 * sum(lat) / len(lat),
        "wall_s": t_last - t_first,
        "term_products_per_s": sum(term_products[k] for k in ok) / max(t_last - t_first, 1e-9),
        "requests": len(requests),
        "failed": len(requests) - len(ok),
        "state": state,
    }
