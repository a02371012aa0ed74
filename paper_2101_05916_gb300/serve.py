"""Trace replay against the continuous-batching server.

A submitter thread replays request arrival times in wall-clock time: it
sleeps until each arrival, then submits through the hj_server_* C ABI.  The
server's worker thread, inside libhj_gb300.so, admits requests under the
HBM budget and steps them together on the GPU.  A collector waits for every
ticket.  For comparison, `replay_fifo_cold` serves the same trace the plain
way: one cold single-grid hj_solve at a time, in arrival order.
"""
from __future__ import annotations

import threading
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import hj

# subsystem keys for warm-start residency: one resident prior per type and grid
_KEYS: Dict[tuple, int] = {}


def request_key(spec) -> int:
    k = (spec.model, spec.n, spec.name)
    if k not in _KEYS:
        _KEYS[k] = len(_KEYS) + 1
    return _KEYS[k]


def shard(trace: Sequence, rank: int, world: int) -> List:
    """Requests of one rank when a trace is spread over `world` independent
    GPUs: round-robin by arrival order, no data exchanged between ranks."""
    return [r for i, r in enumerate(trace) if i % world == rank]


def solve_opts_for(req) -> Dict:
    """Stop rule per subsystem type (see scenarios.X4_OPTS / Z_OPTS)."""
    from .scenarios import X4_OPTS, Z_OPTS
    base = X4_OPTS if req.spec.ndim == 4 else Z_OPTS
    return dict(base, scheme=req.scheme)


def replay_server(trace: Sequence, budget_bytes: int = 40 << 30, max_active: int = 64,
                  time_scale: float = 1.0, warm: bool = True, stream=None,
                  order: int = hj.HJ_ORDER_SHORTEST, max_active_nodes: int = 6_000_000,
                  coarse_4d: int = 0, coarse_levels: int = 1, coarse_scheme: int = 0,
                  keep_values: bool = False) -> Dict:
    """Replay `trace` (workloads.Request list); returns latency stats.

    Default policy: shortest estimated work first, at most 6M nodes of large
    grids stepping at once (small grids ride along).  coarse_4d > 0 runs every
    4-D request with coarse initialisation (Sec. III-C) on a grid of
    max(coarse_4d, n/2) nodes per axis: exact or conservative, far fewer fine
    steps.  coarse_levels = 2 adds a coarser level of max(9, n/4) nodes below
    it; coarse_scheme sets the coarse levels' scheme (0: the request's).
    keep_values: each request's result is copied into a device tensor
    (returned under "values", in trace order) before its ticket is released."""
    s = hj.hj_server_create(budget_bytes, max_active, stream)
    hj.hj_server_set_policy(s, order, max_active_nodes)
    tickets: List[int] = [0] * len(trace)
    t0 = time.perf_counter()

    def submit():
        for i, r in enumerate(trace):
            delay = r.arrival_s * time_scale - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            cn, cn2 = 0, 0
            if coarse_4d and r.spec.ndim == 4:
                cn = max(coarse_4d, min(r.spec.n) // 2)
                cn = cn if cn < min(r.spec.n) else 0
                if cn and coarse_levels == 2 and max(9, min(r.spec.n) // 4) < cn:
                    cn, cn2 = max(9, min(r.spec.n) // 4), cn
            req = hj.make_request(r.spec, hj.HJ_WARM if warm else hj.HJ_COLD,
                                  request_key(r.spec), coarse_n=cn, coarse_n2=cn2,
                                  coarse_scheme=coarse_scheme, **solve_opts_for(r))
            tickets[i] = hj.hj_server_submit(s, req)

    th = threading.Thread(target=submit)
    th.start()
    th.join()
    lat, statuses, steps, values = [], [], [], []
    for r, t in zip(trace, tickets):
        rc, st = hj.hj_server_wait(s, t)
        statuses.append(rc)
        lat.append(st["wall_ms"])
        steps.append(st["steps"])
        if keep_values:
            import torch
            v = torch.empty(r.spec.npts, dtype=torch.float32, device="cuda")
            hj.hj_server_get_value(s, t, v)
            values.append(v)
        hj.hj_server_release(s, t)
    stats = hj.hj_server_get_stats(s)
    hj.hj_server_destroy(s)
    wall = time.perf_counter() - t0
    return dict(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(np.mean(lat)), wall_s=wall, statuses=statuses,
                updates=stats["updates"], updates_per_s=stats["updates"] / max(wall, 1e-9),
                server=stats, latencies_ms=lat, steps=steps, values=values)


def replay_fifo_cold(trace: Sequence, time_scale: float = 1.0, stream=None,
                     check: Optional[Dict[str, List]] = None) -> Dict:
    """The plain baseline: each request solved cold on its own grid, one at a
    time, in arrival order; latency = completion - arrival.

    check: {form name: per-request device tensors of another way of serving
    the same trace}.  Each of them is compared node by node with the cold
    result of its request (scenarios.accuracy) right after that request's
    solve, outside the latency clock; the results come back under
    "accuracy"."""
    from .scenarios import _acc
    t0 = time.perf_counter()
    lat, updates, statuses = [], 0.0, []
    acc = {k: [] for k in (check or {})}
    paused = 0.0
    for i, r in enumerate(trace):
        arrive = r.arrival_s * time_scale
        now = time.perf_counter() - t0 - paused
        if arrive > now:
            time.sleep(arrive - now)
        g = hj.Grid.from_spec(r.spec, stream=stream)
        opts = solve_opts_for(r)
        rc, st = hj.hj_solve(g.handle, hj.HJ_COLD, hj.make_opts(**opts), raise_on_error=False)
        done = time.perf_counter() - t0 - paused
        if check:
            # the comparison is not part of the plain way's latency: its
            # time is taken off the clock
            p0 = time.perf_counter()
            import torch
            v = torch.empty(r.spec.npts, dtype=torch.float32, device="cuda")
            g.value_into(v)
            for name, vals in check.items():
                acc[name].append(_acc(vals[i].reshape(r.spec.n), v.reshape(r.spec.n), r.spec))
            paused += time.perf_counter() - p0
        g.close()
        lat.append(1e3 * (done - arrive))
        updates += float(r.spec.npts) * st["steps"]
        statuses.append(rc)
    wall = time.perf_counter() - t0 - paused
    return dict(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(np.mean(lat)), wall_s=wall, statuses=statuses, updates=updates,
                updates_per_s=updates / max(wall, 1e-9), latencies_ms=lat, accuracy=acc)


def main(argv=None) -> None:
    """python -m paper_2101_05916_gb300.serve [--requests K] [--coarse N] [--no-plain]

    Replays the first K requests of the seeded serving trace through the
    server and through one-at-a-time cold solves; prints one JSON line."""
    import argparse
    import json

    from . import build, workloads as wl
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--coarse", type=int, default=0,
                    help="coarse initialisation of the 4-D requests (nodes per axis, 0 = off)")
    ap.add_argument("--no-plain", action="store_true")
    a = ap.parse_args(argv)
    build.build()
    trace = wl.serving_trace()[:a.requests]
    keep = ("p50_ms", "p99_ms", "mean_ms", "wall_s", "updates_per_s", "updates")
    s = replay_server(trace, coarse_4d=a.coarse)
    out = {"requests": len(trace), "coarse_4d": a.coarse, "served": {k: s[k] for k in keep},
           "server_stats": s["server"], "served_statuses": sorted(set(s["statuses"]))}
    if not a.no_plain:
        p = replay_fifo_cold(trace)
        out["plain_cold"] = {k: p[k] for k in keep}
        out["plain_statuses"] = sorted(set(p["statuses"]))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
