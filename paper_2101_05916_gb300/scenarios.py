"""End-to-end scenarios of the safe-set update method, measured on the GPU.

Each scenario runs the paper's accelerations against the plain way of
solving, through the same C ABI:

* decomposed_update (Sec. III-A + III-B): the x, y and z subsystems of the
  10-D quadcopter.  After every new wind bound they are solved as one batch,
  warm-started from the previous fixed point.  The plain way is three cold
  single-grid solves, one after another.
* adaptive_grid (Sec. III-C): a coarse cold solve, migration to the fine
  grid, and a warm fine solve.  The plain way is a cold fine solve.
* serving: a seeded request trace replayed through the continuous-batching
  server.  The plain way is one cold single-grid solve per request, in
  arrival order.

All times are wall-clock milliseconds of the calls, with the inputs already
on the device.
"""
from __future__ import annotations

import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import hj, serve
from . import workloads as wl

# Solve settings of the 4-D x/y subsystems on truncated grids: the monotone
# clamp min(W3, l, W_prev) ("the tube stays monotone") and a stop test on the
# band |W| <= 0.5 around the zero level set.  With the variational-inequality
# clamp alone, high-order stencils keep cycling at the faces where
# trajectories leave the grid; the monotone clamp keeps the downswings, which
# gives a conservative safe set and convergence on every seeded request.
X4_OPTS = dict(scheme=hj.HJ_WENO5, clamp=hj.HJ_CLAMP_MONOTONE, band=0.5, max_steps=200000,
               max_wall_ms=300000.0)
Z_OPTS = dict(scheme=hj.HJ_ENO2, clamp=hj.HJ_CLAMP_VI, band=0.0, max_steps=200000,
              max_wall_ms=300000.0)


def _opts_for(spec) -> Dict:
    return X4_OPTS if spec.ndim == 4 else Z_OPTS


def _sync():
    import torch
    torch.cuda.synchronize()


def decomposed_update(n4: int = 61, n2: int = 201,
                      bounds: Sequence[float] = wl.CONFIG2_BOUNDS) -> Dict:
    """Wind bound raised in sequence; every update of {x, y, z} is one batch
    warm-started from the previous fixed points (a larger wind bound with the
    same constraint keeps the prior dominating, so the warm start is exact).
    Baseline: cold single-grid solves of x, y and z in turn."""
    specs = wl.config2(n4, n2)
    grids = [hj.Grid.from_spec(s) for s in specs]
    opts = [hj.make_opts(**_opts_for(s)) for s in specs]
    batched: List[Dict] = []
    for k, b in enumerate(bounds):
        for g, s in zip(grids, specs):
            g.set_disturbance_bound([-b] * len(s.d_lo), [b] * len(s.d_hi))
        modes = [hj.HJ_COLD if k == 0 else hj.HJ_WARM] * len(grids)
        _sync()
        t0 = time.perf_counter()
        rc, sts, stats = hj.hj_solve_batch([g.handle for g in grids], modes, opts)
        _sync()
        ms = 1e3 * (time.perf_counter() - t0)
        batched.append(dict(bound=b, ms=ms, steps=[s["steps"] for s in stats],
                            statuses=sts, mode="cold" if k == 0 else "warm"))
    safe = [float(np.mean(g.value() >= 0)) for g in grids]
    finals = [g.value() for g in grids]
    for g in grids:
        g.close()
    plain: List[Dict] = []
    for b in bounds[1:]:
        total, steps, rcs = 0.0, [], []
        outs = []
        for s in specs:
            g = hj.Grid.from_spec(s.with_bound(b))
            _sync()
            t0 = time.perf_counter()
            rc, st = hj.hj_solve(g.handle, hj.HJ_COLD, hj.make_opts(**_opts_for(s)),
                                 raise_on_error=False)
            _sync()
            total += 1e3 * (time.perf_counter() - t0)
            steps.append(st["steps"])
            rcs.append(rc)
            outs.append(g.value())
            g.close()
        plain.append(dict(bound=b, ms=total, steps=steps, statuses=rcs))
    # the last warm batch against the last cold solves
    sign_agree = [float(np.mean((a >= 0) == (c >= 0))) for a, c in zip(finals, outs)]
    upd = [r["ms"] for r in batched[1:]]
    base = [r["ms"] for r in plain]
    return dict(grids=[s.name + "%s" % (s.n,) for s in specs], batched=batched, plain=plain,
                update_ms_p50=float(np.percentile(upd, 50)),
                update_ms_max=float(np.max(upd)),
                plain_ms_p50=float(np.percentile(base, 50)),
                plain_ms_max=float(np.max(base)),
                safe_fraction=safe, sign_agreement_last_update=sign_agree)


def adaptive_grid(nc: int = 31, nf: int = 81, b: float = 1.0,
                  reference: Optional[Dict] = None) -> Dict:
    """Coarse solve -> multilinear migration -> warm fine solve (Sec. III-C),
    against a cold fine solve.  With `reference` (41^4 oracle samples:
    indices and values), the fine results restricted to every second node
    are compared with it.  That only holds when nf = 81, since 80 = 2 * 40."""
    cs, fs = wl.quad_x4(nc, b), wl.quad_x4(nf, b)
    gc, gf = hj.Grid.from_spec(cs), hj.Grid.from_spec(fs)
    _sync()
    t0 = time.perf_counter()
    stc = gc.solve(hj.HJ_COLD, **X4_OPTS)
    t1 = time.perf_counter()
    hj.prolong(gc, gf)
    _sync()
    t2 = time.perf_counter()
    stw = gf.solve(hj.HJ_WARM, **X4_OPTS)
    _sync()
    t3 = time.perf_counter()
    Ww = gf.value()
    stf = gf.solve(hj.HJ_COLD, **X4_OPTS)
    _sync()
    t4 = time.perf_counter()
    Wc = gf.value()
    gc.close()
    gf.close()
    out = dict(coarse=dict(n=nc, ms=1e3 * (t1 - t0), steps=stc["steps"]),
               prolong_ms=1e3 * (t2 - t1),
               fine_warm=dict(n=nf, ms=1e3 * (t3 - t2), steps=stw["steps"],
                              converged=bool(stw["converged"])),
               fine_cold=dict(n=nf, ms=1e3 * (t4 - t3), steps=stf["steps"],
                              converged=bool(stf["converged"])),
               adaptive_total_ms=1e3 * (t3 - t0),
               sign_agreement=float(np.mean((Ww >= 0) == (Wc >= 0))),
               safe_fraction_adaptive=float(np.mean(Ww >= 0)),
               safe_fraction_cold=float(np.mean(Wc >= 0)),
               max_abs_diff_in_band=float(np.abs(Ww - Wc)[np.abs(Wc) <= 0.5].max()))
    if reference is not None and (nf - 1) % 40 == 0:
        r = (nf - 1) // 40
        idx = reference["idx"] * r
        ref = reference["W"]
        for name, W in (("adaptive", Ww), ("cold", Wc)):
            v = W[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]].astype(np.float64)
            band = np.abs(ref) <= 0.5
            out["vs_oracle41_" + name] = dict(
                max_abs=float(np.abs(v - ref).max()),
                max_abs_in_band=float(np.abs(v - ref)[band].max()) if band.any() else None,
                mean_abs=float(np.abs(v - ref).mean()),
                sign_agreement=float(np.mean((v >= 0) == (ref >= 0))))
    return out


def load_reference(path: str) -> Optional[Dict]:
    """41^4 oracle samples written by tests/golden/make_x41_reference.py."""
    try:
        a = np.loadtxt(path, comments="#")
    except OSError:
        return None
    return dict(idx=a[:, :4].astype(np.int64), W=a[:, 4])


def serving(count: int = 16) -> Dict:
    """The first `count` requests of the seeded serving trace through the
    server (default policy) and through one-at-a-time cold solves."""
    trace = wl.serving_trace()[:count]
    a = serve.replay_server(trace)
    b = serve.replay_fifo_cold(trace)
    keep = ("p50_ms", "p99_ms", "mean_ms", "wall_s", "updates_per_s")
    return dict(requests=count,
                served={k: a[k] for k in keep},
                plain_cold={k: b[k] for k in keep},
                all_converged=all(s == 0 for s in a["statuses"] + b["statuses"]))
