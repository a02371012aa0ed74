"""End-to-end scenarios of the safe-set update method, measured on the GPU.

Each scenario runs the paper's accelerations against the plain way of
solving, through the same C ABI:

* decomposed_update (Sec. III-A, III-B, III-C): the x, y and z subsystems of
  the 10-D quadcopter, updated after every new wind bound.  Variants: one
  warm-started batch; or a coarse warm batch, migration, and a fine batch.
  The plain way is three cold single-grid solves, one after another.
* adaptive_grid (Sec. III-C): a coarse cold solve, migration to the fine
  grid, and a warm fine solve.  The plain way is a cold fine solve.
* local_wind_update (Sec. II-C, III-B): the wind bound rises near one
  place only; warm start from the previous result against a cold solve.
* moving_constraint: the box moves along the position axis; warm start from
  the translated prior against a cold solve.
* safety_filter (Sec. II-A, II-B): the decomposed 10-D filter, batch
  throughput and single-state latency.
* serving: a seeded request trace replayed through the continuous-batching
  server.  The plain way is one cold single-grid solve per request, in
  arrival order.

All times are wall-clock milliseconds of the calls, with the inputs already
on the device.
"""
from __future__ import annotations

import time
from typing import Dict, Optional, Sequence

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


# The accuracy bar of a safe-set update: every node within 1e-4 max|W| of
# the reference value, or below it (conservative: a smaller safe set, which
# Sec. III-B and III-C allow), and the sign of W the same at >= 99.99 % of the
# nodes more than one cell from the reference's zero level set.
ACC_REL = 1e-4
ACC_SIGN = 0.9999


def far_from_zero_level(W):
    """Nodes whose every axis neighbour has the node's sign (W >= 0 or < 0),
    excluding W == 0: the nodes more than one cell from the zero level set.
    W is a torch tensor (any device) or a numpy array."""
    import torch
    t = torch.as_tensor(W)
    pos = t >= 0
    near = torch.zeros_like(pos)
    for ax in range(t.ndim):
        n = t.shape[ax]
        a, b = pos.narrow(ax, 0, n - 1), pos.narrow(ax, 1, n - 1)
        diff = a != b
        near.narrow(ax, 0, n - 1).logical_or_(diff)
        near.narrow(ax, 1, n - 1).logical_or_(diff)
    return ~near & (t != 0)


def accuracy(W_fast, W_ref, rel: float = ACC_REL, sign_frac: float = ACC_SIGN,
             band: float = 0.0, margin: int = 0, margin_axes: Sequence[int] = ()) -> Dict:
    """Node-by-node check of an accelerated result W_fast against the
    reference W_ref on the same grid (torch tensors or numpy arrays).

    exact: max|W_fast - W_ref| <= rel max|W_ref|.  conservative: W_fast <=
    W_ref + rel max|W_ref| everywhere.  meets_bar: conservative and the sign
    agreement away from the zero level set is at least sign_frac.  All of
    these are over every node.

    With band > 0 the same value checks are also reported (suffix _watched)
    over the nodes a band stop test watches: |W_ref| <= band, and, with
    margin > 0, farther than margin cells from both faces of every axis in
    margin_axes.  Outside them no stop test has certified either value."""
    import torch
    a = torch.as_tensor(W_fast).to(torch.float64)
    b = torch.as_tensor(W_ref).to(a.device, torch.float64).reshape(a.shape)
    scale = float(b.abs().max())
    d = a - b
    far = far_from_zero_level(b)
    nfar = int(far.sum())
    agree = float(((a >= 0) == (b >= 0))[far].double().mean()) if nfar else 1.0
    excess = float(d.max())
    max_abs = float(d.abs().max())
    tol = rel * scale
    out = dict(max_abs=max_abs, max_excess=excess, scale=scale, sign_agreement_far=agree,
               exact=max_abs <= tol, conservative=excess <= tol)
    out["meets_bar"] = bool(out["conservative"] and agree >= sign_frac)
    if band > 0.0:
        w = b.abs() <= band
        for ax in (margin_axes if margin > 0 else ()):
            n = b.shape[ax]
            i = torch.arange(n, device=b.device)
            keep = (i >= margin) & (i <= n - 1 - margin)
            shape = [1] * b.ndim
            shape[ax] = n
            w = w & keep.view(shape)
        if bool(w.any()):
            dw = d[w]
            out.update(max_abs_watched=float(dw.abs().max()), max_excess_watched=float(dw.max()),
                       exact_watched=float(dw.abs().max()) <= tol,
                       conservative_watched=float(dw.max()) <= tol)
            out["meets_bar_watched"] = bool(out["conservative_watched"] and agree >= sign_frac)
    return out


def _opts_for(spec) -> Dict:
    return X4_OPTS if spec.ndim == 4 else Z_OPTS


def _acc(W_fast, W_ref, spec) -> Dict:
    """accuracy() with the band of the spec's stop test reported as well."""
    o = _opts_for(spec)
    return accuracy(W_fast, W_ref, band=o.get("band", 0.0), margin=o.get("band_margin", 0),
                    margin_axes=tuple(range(1, spec.ndim)))


def _sync():
    import torch
    torch.cuda.synchronize()


def _batch(grids, modes, specs):
    opts = [hj.make_opts(**_opts_for(s)) for s in specs]
    _sync()
    t0 = time.perf_counter()
    rc, sts, stats = hj.hj_solve_batch([g.handle for g in grids], modes, opts)
    _sync()
    return 1e3 * (time.perf_counter() - t0), [s["steps"] for s in stats], sts


def decomposed_update(n4: int = 61, n2: int = 201, nc4: int = 31, nc2: int = 101,
                      bounds: Sequence[float] = wl.CONFIG2_BOUNDS) -> Dict:
    """The wind bound is raised in sequence.  Every update of {x, y, z} is
    solved three ways, as in the three columns of the paper's Table I:

    * plain: cold single-grid solves of x, y and z in turn (decomposition
      only);
    * warm: one batch of the three grids, warm-started from the previous fixed
      points (decomposition + warm start).  A larger bound with the same
      constraint keeps the prior dominating;
    * new: the coarse grids (x, y at nc4^4, z at nc2^2) solved as one batch,
      warm from their previous fixed points, then migrated to the fine grids,
      which are solved as one batch from the migrated values (decomposition +
      warm start + coarse initialization, Sec. III-C).
    """
    specs = wl.config2(n4, n2)
    coarse_specs = wl.config2(nc4, nc2)
    warm_grids = [hj.Grid.from_spec(s) for s in specs]
    fine = [hj.Grid.from_spec(s) for s in specs]
    coarse = [hj.Grid.from_spec(s) for s in coarse_specs]
    rows = []
    for k, b in enumerate(bounds):
        for g, s in zip(warm_grids + fine, specs + specs):
            g.set_disturbance_bound([-b] * len(s.d_lo), [b] * len(s.d_hi))
        for g, s in zip(coarse, coarse_specs):
            g.set_disturbance_bound([-b] * len(s.d_lo), [b] * len(s.d_hi))
        first = k == 0
        w_ms, w_steps, w_sts = _batch(warm_grids, [hj.HJ_COLD if first else hj.HJ_WARM] * 3, specs)
        c_ms, c_steps, c_sts = _batch(coarse, [hj.HJ_COLD if first else hj.HJ_WARM] * 3,
                                      coarse_specs)
        _sync()
        t0 = time.perf_counter()
        for gc, gf in zip(coarse, fine):
            hj.prolong(gc, gf)
        _sync()
        p_ms = 1e3 * (time.perf_counter() - t0)
        f_ms, f_steps, f_sts = _batch(fine, [hj.HJ_WARM] * 3, specs)
        row = dict(bound=b, warm_ms=w_ms, warm_steps=w_steps, new_ms=c_ms + p_ms + f_ms,
                   new_coarse_steps=c_steps, new_fine_steps=f_steps,
                   statuses=[int(x) for x in w_sts + c_sts + f_sts])
        if not first:
            total, steps, outs = 0.0, [], []
            for s in specs:
                g = hj.Grid.from_spec(s.with_bound(b))
                _sync()
                t1 = time.perf_counter()
                rc, st = hj.hj_solve(g.handle, hj.HJ_COLD, hj.make_opts(**_opts_for(s)),
                                     raise_on_error=False)
                _sync()
                total += 1e3 * (time.perf_counter() - t1)
                steps.append(st["steps"])
                outs.append(g.value())
                g.close()
            row.update(plain_ms=total, plain_steps=steps)
            row["accuracy_warm"] = [_acc(g.value(), c, sp)
                                    for g, c, sp in zip(warm_grids, outs, specs)]
            row["accuracy_new"] = [_acc(g.value(), c, sp) for g, c, sp in zip(fine, outs, specs)]
            row["warm_meets_bar"] = all(a["meets_bar"] for a in row["accuracy_warm"])
            row["new_meets_bar"] = all(a["meets_bar"] for a in row["accuracy_new"])
        rows.append(row)
    for g in warm_grids + fine + coarse:
        g.close()
    upd = rows[1:]

    def p50(key):
        return float(np.percentile([r[key] for r in upd], 50))

    return dict(grids=[s.name + "%s" % (s.n,) for s in specs],
                coarse_grids=[s.name + "%s" % (s.n,) for s in coarse_specs], updates=rows,
                plain_ms_p50=p50("plain_ms"), warm_ms_p50=p50("warm_ms"), new_ms_p50=p50("new_ms"),
                speedup_new_vs_plain=p50("plain_ms") / p50("new_ms"),
                warm_meets_bar=all(r["warm_meets_bar"] for r in upd),
                new_meets_bar=all(r["new_meets_bar"] for r in upd))


def adaptive_grid(nc: int = 31, nf: int = 81, b: float = 1.0,
                  reference: Optional[Dict] = None,
                  variants: Sequence[tuple] = (((41,), 0), ((21, 41), 0), ((31,), 2),
                                               ((21, 41), 2))) -> Dict:
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
    # more levels, and cheap gradients (ENO2) on the coarse levels
    levels_out = []
    for levels, coarse_scheme in variants:
        grids = [hj.Grid.from_spec(wl.quad_x4(n, b)) for n in tuple(levels) + (nf,)]
        _sync()
        t5 = time.perf_counter()
        steps = []
        for k, g in enumerate(grids):
            opts = dict(X4_OPTS)
            if k < len(levels) and coarse_scheme:
                opts["scheme"] = coarse_scheme
            if k:
                hj.prolong(grids[k - 1], g)
            steps.append(g.solve(hj.HJ_WARM if k else hj.HJ_COLD, **opts)["steps"])
        _sync()
        ms = 1e3 * (time.perf_counter() - t5)
        Wv = grids[-1].value()
        for g in grids:
            g.close()
        levels_out.append(dict(levels=list(levels) + [nf],
                               coarse_scheme="ENO2" if coarse_scheme == 2 else "WENO5",
                               ms=ms, steps=steps, speedup_vs_cold=1e3 * (t4 - t3) / ms,
                               accuracy=_acc(Wv, Wc, fs),
                               sign_agreement=float(np.mean((Wv >= 0) == (Wc >= 0))),
                               max_abs_diff_in_band=float(
                                   np.abs(Wv - Wc)[np.abs(Wc) <= 0.5].max())))
    out = dict(coarse=dict(n=nc, ms=1e3 * (t1 - t0), steps=stc["steps"]),
               prolong_ms=1e3 * (t2 - t1),
               fine_warm=dict(n=nf, ms=1e3 * (t3 - t2), steps=stw["steps"],
                              converged=bool(stw["converged"])),
               fine_cold=dict(n=nf, ms=1e3 * (t4 - t3), steps=stf["steps"],
                              converged=bool(stf["converged"])),
               adaptive_total_ms=1e3 * (t3 - t0),
               accuracy=_acc(Ww, Wc, fs),
               sign_agreement=float(np.mean((Ww >= 0) == (Wc >= 0))),
               safe_fraction_adaptive=float(np.mean(Ww >= 0)),
               safe_fraction_cold=float(np.mean(Wc >= 0)),
               max_abs_diff_in_band=float(np.abs(Ww - Wc)[np.abs(Wc) <= 0.5].max()),
               levels=levels_out)
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


def local_wind_update(n4: int = 61, n2: int = 201, base: float = 0.5,
                      bumps: Sequence[tuple] = ((0.5, 3.0, 0.6), (0.5, -2.5, 0.6),
                                                (0.8, 3.2, 0.4))) -> Dict:
    """State-dependent wind (Sec. II-C, V-A): the GP learns that the wind is
    stronger near one place, so the bound rises locally.  Each bump
    (height, centre on the position axis, width) is added to the previous
    field, so the previous fixed point dominates the new one and the warm
    start stays exact (Sec. III-B).  Every update of the x (n4^4) and z
    (n2^2) subsystems is solved warm from the previous result and cold."""
    specs = [wl.quad_x4(n4, base), wl.quad_z(n2, base)]
    rows = []
    for spec in specs:
        opts = hj.make_opts(**_opts_for(spec))
        g = hj.Grid.from_spec(spec)
        lo, hi = wl.wind_field(spec, base, 0.0, 0, 0.0, 1.0)
        g.set_disturbance_field(lo, hi)
        rc, st = hj.hj_solve(g.handle, hj.HJ_COLD, opts, raise_on_error=False)
        for height, centre, width in bumps:
            # the z axis spans [0, 3]: put its bumps at the same relative place
            c = centre if spec.ndim == 4 else 1.5 + 0.3 * centre
            w = width if spec.ndim == 4 else 0.3 * width
            dlo, dhi = wl.wind_field(spec, 0.0, height, 0, c, w)
            lo, hi = lo + dlo, hi + dhi
            g.set_disturbance_field(lo, hi)
            _sync()
            t0 = time.perf_counter()
            rcw, stw = hj.hj_solve(g.handle, hj.HJ_WARM, opts, raise_on_error=False)
            _sync()
            t1 = time.perf_counter()
            Ww = g.value()
            gc = hj.Grid.from_spec(spec)
            gc.set_disturbance_field(lo, hi)
            _sync()
            t2 = time.perf_counter()
            rcc, stc = hj.hj_solve(gc.handle, hj.HJ_COLD, opts, raise_on_error=False)
            _sync()
            t3 = time.perf_counter()
            Wc = gc.value()
            gc.close()
            rows.append(dict(grid=spec.name + "%s" % (spec.n,), bump=(height, c, w),
                             warm_ms=1e3 * (t1 - t0), warm_steps=stw["steps"],
                             cold_ms=1e3 * (t3 - t2), cold_steps=stc["steps"],
                             statuses=[int(rcw), int(rcc)], accuracy=_acc(Ww, Wc, spec),
                             sign_agreement=float(np.mean((Ww >= 0) == (Wc >= 0))),
                             max_abs_diff_in_band=float(
                                 np.abs(Ww - Wc)[np.abs(Wc) <= 0.5].max())))
        g.close()
    speed = [r["cold_ms"] / r["warm_ms"] for r in rows]
    return dict(base=base, updates=rows, warm_speedup_p50=float(np.percentile(speed, 50)),
                meets_bar=[r["grid"] for r in rows if r["accuracy"]["meets_bar"]])


# The exact 4-D setting (Sec. II-A's Eq. 2 clamp): VI clamp, band stop test
# that skips a 6-cell layer at the faces of the free axes.  Warm and cold
# solves agree here; the monotone clamp's do not.
X4_EXACT_OPTS = dict(scheme=hj.HJ_WENO5, clamp=hj.HJ_CLAMP_VI, band=0.5, band_margin=6,
                     max_steps=200000, max_wall_ms=300000.0)


def localized_update(n4: int = 61, base: float = 0.5, local_tol: float = 1e-6,
                     bumps: Sequence[tuple] = ((0.5, 3.0, 0.6), (0.5, -2.5, 0.6),
                                               (0.8, 3.2, 0.4))) -> Dict:
    """Localized warm starting (Sec. VI) on the exact 4-D setting: the wind
    bound of the x subsystem (n4^4) rises near one place, three times in a
    row (each bump added to the previous field, so every prior dominates).
    Each update is solved three ways from the same state: cold, warm from the
    previous result, and warm with localized stepping (local_tol).  Each
    result is checked node by node against the cold one (accuracy, also on
    the watched nodes of the stop test)."""
    spec = wl.quad_x4(n4, base)
    opts = hj.make_opts(**X4_EXACT_OPTS)
    lopts = hj.make_opts(local_tol=local_tol, **X4_EXACT_OPTS)
    import torch
    g = hj.Grid.from_spec(spec)
    lo, hi = wl.wind_field(spec, base, 0.0, 0, 0.0, 1.0)
    g.set_disturbance_field(lo, hi)
    hj.hj_solve(g.handle, hj.HJ_COLD, opts, raise_on_error=False)
    prior = torch.empty(spec.npts, dtype=torch.float32, device="cuda")
    rows = []
    for height, centre, width in bumps:
        g.value_into(prior)
        dlo, dhi = wl.wind_field(spec, 0.0, height, 0, centre, width)
        lo, hi = lo + dlo, hi + dhi
        g.set_disturbance_field(lo, hi)
        runs = {}
        for name, mode, o in (("cold", hj.HJ_COLD, opts), ("warm", hj.HJ_WARM, opts),
                              ("local", hj.HJ_WARM, lopts)):
            g.set_value(prior)
            _sync()
            t0 = time.perf_counter()
            rc, st = hj.hj_solve(g.handle, mode, o, raise_on_error=False)
            _sync()
            ms = 1e3 * (time.perf_counter() - t0)
            W = torch.empty(spec.npts, dtype=torch.float32, device="cuda")
            g.value_into(W)
            runs[name] = (ms, st, rc, W.reshape(spec.n))
        # continue the sequence from the localized result
        g.set_value(runs["local"][3].reshape(-1))
        row = dict(bump=(height, centre, width))
        for name, (ms, st, rc, W) in runs.items():
            row[name] = dict(ms=ms, steps=st["steps"], stepped=st["stepped"], status=int(rc))
            if name != "cold":
                row[name]["accuracy"] = accuracy(W, runs["cold"][3], band=0.5, margin=6,
                                                 margin_axes=(1, 2, 3))
        rows.append(row)
    g.close()
    sp = [r["cold"]["ms"] / r["local"]["ms"] for r in rows]
    return dict(grid=[n4] * 4, setting="VI clamp, band 0.5, face margin 6", local_tol=local_tol,
                updates=rows, local_speedup_vs_cold_p50=float(np.percentile(sp, 50)),
                local_meets_bar_watched=all(r["local"]["accuracy"].get("meets_bar_watched", False)
                                            for r in rows),
                local_meets_bar=all(r["local"]["accuracy"]["meets_bar"] for r in rows))


def moving_constraint(n4: int = 61, n2: int = 201, b: float = 0.5,
                      shifts: Sequence[float] = (0.25, 0.5, 0.25, -0.25)) -> Dict:
    """The constraint box moves along the position axis (a moving safe
    corridor).  The quadcopter blocks' dynamics do not depend on position,
    so each update warm-starts from the previous fixed point translated by
    the move (hj_translate); the plain way is a cold solve of the moved box.
    x (n4^4) boxes |p - s| <= 4 on [-5, 5]; z (n2^2) boxes [0.5, 2.5] + s/2."""
    rows = []
    for kind in ("x", "z"):
        def spec_at(sh):
            if kind == "x":
                return wl.quad_x4(n4, b, shift=sh)
            return wl.quad_z(n2, b, (0.5 + 0.5 * sh, 2.5 + 0.5 * sh))
        prev_shift = 0.0
        prev = hj.Grid.from_spec(spec_at(0.0))
        opts = hj.make_opts(**_opts_for(prev.spec))
        hj.hj_solve(prev.handle, hj.HJ_COLD, opts, raise_on_error=False)
        for sh in shifts:
            spec = spec_at(sh)
            move = (sh - prev_shift) * (1.0 if kind == "x" else 0.5)
            cur = hj.Grid.from_spec(spec)
            _sync()
            t0 = time.perf_counter()
            hj.translate(prev, cur, [move] + [0.0] * (spec.ndim - 1))
            rcw, stw = hj.hj_solve(cur.handle, hj.HJ_WARM, opts, raise_on_error=False)
            _sync()
            t1 = time.perf_counter()
            Ww = cur.value()
            cold = hj.Grid.from_spec(spec)
            _sync()
            t2 = time.perf_counter()
            rcc, stc = hj.hj_solve(cold.handle, hj.HJ_COLD, opts, raise_on_error=False)
            _sync()
            t3 = time.perf_counter()
            Wc = cold.value()
            cold.close()
            rows.append(dict(grid=spec.name + "%s" % (spec.n,), move=move,
                             translated_warm_ms=1e3 * (t1 - t0), warm_steps=stw["steps"],
                             cold_ms=1e3 * (t3 - t2), cold_steps=stc["steps"],
                             statuses=[int(rcw), int(rcc)], accuracy=_acc(Ww, Wc, spec),
                             sign_agreement=float(np.mean((Ww >= 0) == (Wc >= 0))),
                             max_abs_diff_in_band=float(
                                 np.abs(Ww - Wc)[np.abs(Wc) <= 0.5].max())))
            prev.close()
            prev, prev_shift = cur, sh
        prev.close()
    speed = [r["cold_ms"] / r["translated_warm_ms"] for r in rows]
    return dict(updates=rows, speedup_p50=float(np.percentile(speed, 50)),
                meets_bar=[(r["grid"], r["move"]) for r in rows if r["accuracy"]["meets_bar"]])


def safety_filter(n4: int = 41, n2: int = 201, batch: int = 1 << 20, reps: int = 20,
                  single: int = 200) -> Dict:
    """The decomposed 10-D safety filter (Sec. II-A, II-B, III-A) over the x,
    y (n4^4) and z (n2^2) subsystems of the 10-D demo: throughput for a batch
    of states resident on the device, and the latency of one state through
    host buffers, as a control loop would call it."""
    import torch
    specs = [wl.demo10d_x(n4, 0.5), wl.demo10d_x(n4, 0.5, "y"), wl.demo10d_z(n2, 0.5)]
    grids = [hj.Grid.from_spec(s) for s in specs]
    for g, s in zip(grids, specs):
        g.solve(hj.HJ_COLD, **_opts_for(s))
    states = wl.quad10d_states(specs, batch, seed=5)
    up = np.tile([0.0, 0.0, 9.81 / 0.91], (batch, 1))
    ts, tu = torch.from_numpy(states).cuda(), torch.from_numpy(up).cuda()
    hj.hj_safety_filter(grids, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, ts, tu, 0.0)
    _sync()
    t0 = time.perf_counter()
    for _ in range(reps):
        u, w, act = hj.hj_safety_filter(grids, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, ts, tu, 0.0)
    _sync()
    dt_batch = (time.perf_counter() - t0) / reps
    active = float((act != 0).float().mean().item())
    one_x, one_u = states[:1].copy(), up[:1].copy()
    filt = hj.SafetyFilter(grids, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, 10, 3)
    filt(one_x, one_u, 0.0)
    lat = []
    for i in range(single):
        one_x[0] = states[i]
        t1 = time.perf_counter()
        filt(one_x, one_u, 0.0)
        lat.append(time.perf_counter() - t1)
    for g in grids:
        g.close()
    return dict(grids=[s.name + "%s" % (s.n,) for s in specs], batch=batch,
                batch_ms=1e3 * dt_batch, states_per_s=batch / dt_batch,
                active_fraction=active,
                single_state_us_p50=1e6 * float(np.percentile(lat, 50)),
                single_state_us_p99=1e6 * float(np.percentile(lat, 99)))


def load_reference(path: str) -> Optional[Dict]:
    """41^4 oracle samples written by tests/golden/make_x41_reference.py."""
    try:
        a = np.loadtxt(path, comments="#")
    except OSError:
        return None
    return dict(idx=a[:, :4].astype(np.int64), W=a[:, 4])


def summarize_accuracy(accs) -> Dict:
    """Per-request accuracy results of one way of serving -> the form's
    verdict: it meets the bar only if every request does."""
    if not accs:
        return dict(requests=0, meets_bar=None)
    ok = [a["meets_bar"] for a in accs]
    okw = [a.get("meets_bar_watched", a["meets_bar"]) for a in accs]
    return dict(requests=len(accs), requests_meeting_bar=int(sum(ok)),
                requests_exact=int(sum(a["exact"] for a in accs)),
                meets_bar=bool(all(ok)),
                requests_meeting_bar_watched=int(sum(okw)), meets_bar_watched=bool(all(okw)),
                worst_sign_agreement_far=float(min(a["sign_agreement_far"] for a in accs)),
                worst_excess_rel=float(max(a["max_excess"] / max(a["scale"], 1e-30)
                                           for a in accs)),
                worst_abs_rel=float(max(a["max_abs"] / max(a["scale"], 1e-30) for a in accs)))


def serving(count: int = 16, coarse_4d: int = 13, forms: Sequence[str] = ("served",
            "served_coarse_init")) -> Dict:
    """The first `count` requests of the seeded serving trace through the
    server and through one-at-a-time cold solves.  Forms: "served" (default
    policy, resident warm starts under the dominance rule),
    "served_coarse_init" (the 4-D requests with coarse initialisation, WENO5
    on the coarse grid) and "served_coarse_init_eno2" (cheap ENO2 gradients
    there).  Every served result is checked node by node against the cold
    solve of its request (accuracy); p50/p99 of a form count as a result
    at the stated accuracy only when all its requests meet the bar."""
    trace = wl.serving_trace()[:count]
    runs = {}
    for f in forms:
        kw = {}
        if f.startswith("served_coarse_init"):
            kw["coarse_4d"] = coarse_4d
        if f == "served_coarse_init_eno2":
            kw["coarse_scheme"] = hj.HJ_ENO2
        runs[f] = serve.replay_server(trace, keep_values=True, **kw)
    b = serve.replay_fifo_cold(trace, check={f: r["values"] for f, r in runs.items()})
    keep = ("p50_ms", "p99_ms", "mean_ms", "wall_s", "updates_per_s")
    out = dict(requests=count, plain_cold={k: b[k] for k in keep})
    statuses = list(b["statuses"])
    for f, r in runs.items():
        out[f] = dict({k: r[k] for k in keep}, accuracy=summarize_accuracy(b["accuracy"][f]))
        statuses += r["statuses"]
        r["values"].clear()
    out["all_converged"] = all(st == 0 for st in statuses)
    out["forms_at_the_bar"] = [f for f in runs if out[f]["accuracy"]["meets_bar"]]
    return out


def warm_start_diagnosis(n: int = 61, b_prior: float = 0.5, b_new: float = 1.0,
                         face: int = 6, max_windows: int = 200, clamp: int = hj.HJ_CLAMP_MONOTONE,
                         band: float = 0.5, tol: float = 1e-4) -> Dict:
    """Where a 4-D update spends its windows.  The x-subsystem (n^4) is solved
    cold at b_prior; then the b_new update is run window by window (0.1 s of
    simulated time each, the stop rule's window), from that prior (warm) and
    from the constraint (cold).  After every window the change since the
    window's start is split by where it sits: the band |W| <= band that the
    stop test watches, and within it the face layer (nodes within `face`
    cells of a face of a free axis v, theta, omega) against the interior.
    Reported per run: the windows to the stop, and per window the band
    residual in the face layer and the interior and the number of band
    nodes that still change by more than tol."""
    import torch
    spec = wl.quad_x4(n, b_prior)
    g = hj.Grid.from_spec(spec)
    g.solve(hj.HJ_COLD, scheme=hj.HJ_WENO5, clamp=clamp, band=band, tol=tol, max_steps=200000)
    prior = torch.empty(spec.npts, dtype=torch.float32, device="cuda")
    g.value_into(prior)
    g.set_disturbance_bound([-b_new], [b_new])
    a = g.alpha()
    h = [(hi - lo) / (m - 1) for lo, hi, m in zip(spec.lo, spec.hi, spec.n)]
    dt = 0.5 / sum(ai / hi for ai, hi in zip(a, h))
    per = hj.cfl_steps(0.1, dt)
    ii = torch.arange(n, device="cuda")
    dist = torch.minimum(ii, n - 1 - ii)
    d4 = torch.minimum(torch.minimum(dist.view(1, n, 1, 1), dist.view(1, 1, n, 1)),
                       dist.view(1, 1, 1, n)).expand(n, n, n, n)
    in_face = d4 < face
    runs = {}
    for mode in ("warm", "cold"):
        if mode == "warm":
            g.set_value(prior)
            W = prior.clone().reshape(spec.n)
        else:
            # the cold start W = l, with l = 4 - |p| the margin to the box |p| <= 4
            x0 = spec.lo[0] + torch.arange(n, device="cuda", dtype=torch.float64) * h[0]
            l0 = (spec.con_b[0] - spec.con_a[0]) / 2 - (x0 - (spec.con_a[0] + spec.con_b[0]) / 2).abs()
            W = l0.float().view(n, 1, 1, 1).expand(n, n, n, n).contiguous()
            g.set_value(W.reshape(-1))
        cur = torch.empty(spec.npts, dtype=torch.float32, device="cuda")
        rows, stop = [], None
        for k in range(max_windows):
            g.solve(hj.HJ_WARM, scheme=hj.HJ_WENO5, dt=dt, fixed_steps=per, clamp=clamp)
            g.value_into(cur)
            Wn = cur.reshape(spec.n)
            r = (Wn - W).abs()
            inb = torch.minimum(Wn.abs(), W.abs()) <= band
            rb = torch.where(inb, r, torch.zeros_like(r))
            rf = float(rb[in_face].max())
            ri = float(rb[~in_face].max())
            big = rb > tol
            rows.append(dict(window=k + 1, band_resid_face=rf, band_resid_interior=ri,
                             band_nodes_over_tol_face=int((big & in_face).sum()),
                             band_nodes_over_tol_interior=int((big & ~in_face).sum()),
                             resid_all=float(r.max())))
            W = Wn.clone()
            if max(rf, ri) < tol:
                stop = k + 1
                break
        # the last windows before the stop: which part held it up
        tail = rows[-min(10, len(rows)):]
        runs[mode] = dict(windows=stop, steps=None if stop is None else stop * per,
                          held_by_face=sum(1 for r in tail
                                           if r["band_resid_face"] >= r["band_resid_interior"]),
                          tail_windows=len(tail),
                          trace=rows[::max(1, len(rows) // 25)] + rows[-3:])
    g.close()
    return dict(grid=[n] * 4, b_prior=b_prior, b_new=b_new, dt=dt, steps_per_window=per,
                face_layer=face, band=band, tol=tol,
                clamp="monotone" if clamp == hj.HJ_CLAMP_MONOTONE else "vi", runs=runs)
