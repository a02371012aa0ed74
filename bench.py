"""Benchmark: HJ grid-point updates/s of the safe-set solve on GB300.

Headline workload: the adaptive-grid safety update of the 4-D x-subsystem
of the decomposed near-hover quadcopter (Sec. III-C), the largest
single-GPU configuration.  One bench step is one update:
    (1) a cold solve on a coarse 31^4 grid, to convergence;
    (2) multilinear migration of the coarse result onto the 81^4 fine grid
        (43.0 M nodes; its four fields take 689 MB, beyond the 129 MB L2);
    (3) a warm fine solve from the migrated value, to convergence.
Wind bound |d| <= 1.0, WENO5 + TVD-RK3, CFL 0.5, clamp min(W3, l, W_prev)
(the monotone tube), stop at an L-inf change below 1e-4 per 0.1 s window on
the band |W| <= 0.5 around the safe-set boundary.
One grid-point update is one node advanced by one full TVD-RK3 step.
value = total updates (coarse and fine) / total device time of the K timed
steps, CUDA events on the solving stream; L2 is also flushed between steps.

Other keys:
  e2e          the same update through the C ABI from a host description of
               the problem: grids created, solved, the fine value read back
               into pinned host memory, grids destroyed, every step.
  latency_ms   p50/p99 of the update against the plain cold 81^4 solve, with
               the node-by-node accuracy check of the update against it.
  roofline     the dominant kernel (the WENO5 stage kernel on the 81^4 grid):
               per-launch device time, the median of repeated fixed-step
               passes timed with CUDA events.
  secondary    the 41^4 cold solve + warm update pair (the 4-D configuration
               with cold vs warm start), with its own rate and roofline.
  scenarios    the decomposed batched update, coarse-to-fine variants, local
               wind rises, a moving constraint, the safety filter, serving.
  cpu_baseline the FP64 oracle on a bounded sample of the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HJ grid-point updates/s; p50/p99 safe-set update latency vs plain cold solve"
UNIT = "grid-point updates/s"
N_COARSE, N_FINE = 31, 81
BOUND = 1.0
N_C1 = 41
BOUND_C1_PRIOR, BOUND_C1 = 0.0, 0.5
BAND = 0.5
MARGIN = 0
CLAMP = 1  # HJ_CLAMP_MONOTONE

# Algorithmic work per grid-point update (one node, one full TVD-RK3 step),
# counted from the discrete operator (FMA = 2 flops, reciprocal = 1).
# WENO5, 4-D: per axis 6 differences + 2 WENO5 evaluations (59 flops each incl.
# the 1/(6h) scale) + Lax-Friedrichs terms (4) = 128; x 4 axes = 512; plus the
# Hamiltonian (14), coordinates (8) and RK combination (4) = 538 per stage;
# stage 3 adds the clamp/margin (10).  3 stages -> 1624 flops.
FLOPS_PER_UPDATE = {("quad_x4", 5): 1624.0}
# Compulsory DRAM bytes per update: stage 1 reads W, writes W1 (8 B); stage 2
# reads W1, W, writes W2 (12 B); stage 3 reads W2, W, writes W (12 B).
BYTES_PER_UPDATE = 32.0
# DRAM bytes (read + write) per stage launch, averaged over stages 1-3, from
# one ncu capture of the stage kernels on the 81^4 grid (three consecutive
# launches of each of two steps, --clock-control none): 307.3, 493.8 and
# 482.8 MB.  Reset to None whenever the stage kernel changes.
STAGE_TRAFFIC_BYTES_81 = 427972352.0
# The same for the 41^4 grid (11.3, 22.6 and 22.6 MB, reads only: the
# 45 MB working set stays in L2 and the writes never reach DRAM).
STAGE_TRAFFIC_BYTES_41 = 18853803.0
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-scenarios", action="store_true",
                    help="skip the decomposed / adaptive-grid / serving scenarios")
    ap.add_argument("--serve-requests", type=int, default=256,
                    help="requests of the seeded serving trace replayed (all 256 by default)")
    ap.add_argument("--serve-coarse", action="store_true",
                    help="also replay the trace with coarse initialisation of the 4-D requests")
    ap.add_argument("--max-wall-ms", type=float, default=300000.0,
                    help="wall-time cap of each headline solve (0: none; for slow profilers)")
    ap.add_argument("--secondary-steps", type=int, default=3,
                    help="timed steps of the 41^4 cold + warm pair")
    ap.add_argument("--only-headline", action="store_true",
                    help="run the warm-up and timed steps of the headline update only "
                         "(no accuracy check, roofline pass, e2e, secondary, scenarios, oracle)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every stage kernel directly instead of replaying captured "
                         "window graphs (the same computation; for per-launch profilers)")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run only this many fixed TVD-RK3 steps on one grid (for ncu)")
    ap.add_argument("--profile-n", type=int, default=N_FINE,
                    help="nodes per axis of the 4-D grid of --profile-steps")
    ap.add_argument("--profile-tile", type=int, default=0,
                    help="row tiles of this many lines in --profile-steps (0: the flat mapping)")
    return ap.parse_args()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ------------------------------------------------------------- distributed

def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- workloads

def arm_config():
    """The workload both arms report: the adaptive 31^4 -> 81^4 update."""
    return {"workload": "x4_adaptive_31^4->81^4_weno5_update", "grid_coarse": [N_COARSE] * 4,
            "grid_fine": [N_FINE] * 4, "scheme": "WENO5", "rk": "TVD-RK3", "cfl": 0.5,
            "tol": 1e-4, "check_dt": 0.1, "stop_band": BAND, "clamp": "monotone",
            "wind": BOUND, "l2": "fine fields (689 MB) exceed L2; also flushed between steps",
            "parallelism": "independent grids per rank"}


def fp32_peak_tflops(peaks):
    """FP32 lanes x 2 flops x SM count x maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0)) if peaks else 2070.0
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, sms, mhz


def stage_launch_seconds(hj, g, stream, steps=40, reps=5):
    """Average device time of one stage launch on grid g: `reps` warm
    passes of `steps` TVD-RK3 steps, each timed alone with CUDA events on
    the grid's stream; the median pass over its 3 * steps stage launches.
    The pass's initialisation kernel and set-up count against the launches,
    so the figure errs high: 12-step passes read 567 us per 81^4 launch,
    40-step passes 562 us.  Differencing a short
    and a long pass read 1-2 % low on GB300: the two passes do not carry
    the same fixed cost."""
    import torch
    per = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.solve(hj.HJ_WARM, scheme=5, fixed_steps=steps, clamp=CLAMP)
        e1.record(stream)
        e1.synchronize()
        per.append(e0.elapsed_time(e1) / 1e3 / (3 * steps))
    return statistics.median(per)


def roofline_entry(hj, npts, per_launch_s, peak, sms, mhz, traffic, kernel, peaks):
    flops_launch = FLOPS_PER_UPDATE[("quad_x4", 5)] / 3.0 * npts
    achieved = flops_launch / per_launch_s / 1e12
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    hbm_gbs = BYTES_PER_UPDATE / 3.0 * npts / per_launch_s / 1e9
    return {
        "bound": "alu", "kernel": kernel,
        "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
        "peak_source": "FP32 lanes x 2 x SMs x max SM clock (%d x %d x 2 x %.0f MHz)"
                       % (sms, FP32_LANES_PER_SM, mhz),
        "per_launch_us": per_launch_s * 1e6,
        "flops_per_update": FLOPS_PER_UPDATE[("quad_x4", 5)],
        "algorithmic_flops_per_launch": flops_launch,
        "traffic": traffic,
        "algorithmic_bytes_per_launch": BYTES_PER_UPDATE / 3.0 * npts,
        "hbm_view": {"achieved_gbs": hbm_gbs, "bytes_per_update": BYTES_PER_UPDATE,
                     "peak_gbs": hbm_peak, "frac": hbm_gbs / hbm_peak,
                     "peak_source": "measured" if peaks else "fallback"},
    }


def kernel_name(hj, n):
    return ("hj_stage_1..3 (stage kernel, WENO5, quad_x4, specialised to the %d^4 shape)" % n
            if hj.hj_jit_kernels() > 0 else "stage_kernel<4,WENO5,quad_x4>")


# ------------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 oracle as the reference arm: each bench step advances a
    bounded sample of the headline workload (one TVD-RK3 step of the fine
    81^4 WENO5 x-subsystem) on the host cores."""
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    from paper_2101_05916_gb300 import workloads as wl
    spec = wl.quad_x4(N_FINE, BOUND)
    dt = oracle.cfl_dt(spec)
    sample_steps = 1
    for _ in range(args.warmup):
        oracle.solve(spec, scheme=5, dt=dt, fixed_steps=sample_steps, clamp=CLAMP)
    t = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.solve(spec, scheme=5, dt=dt, fixed_steps=sample_steps, clamp=CLAMP)
        t += time.perf_counter() - t0
    updates = spec.npts * sample_steps * args.steps
    v = updates / t
    cores = oracle.num_threads()
    sample = "%d TVD-RK3 step of the 81^4 fine grid of the same update per bench step" % sample_steps
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": arm_config(),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%s, %d steps" % (sample, args.steps)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------- gb300 arm

def cpu_baseline():
    """The oracle on all host cores (one TVD-RK3 step of the 81^4 fine grid)
    and on one core (one step of the 41^4 grid, the same operator)."""
    import oracle
    from paper_2101_05916_gb300 import workloads as wl
    spec = wl.quad_x4(N_FINE, BOUND)
    dt = oracle.cfl_dt(spec)
    t0 = time.perf_counter()
    oracle.solve(spec, scheme=5, dt=dt, fixed_steps=1, clamp=CLAMP)
    t = time.perf_counter() - t0
    cores = oracle.num_threads()
    small = wl.quad_x4(N_C1, BOUND)
    dts = oracle.cfl_dt(small)
    try:
        oracle.set_num_threads(1)
        t1 = time.perf_counter()
        oracle.solve(small, scheme=5, dt=dts, fixed_steps=1, clamp=CLAMP)
        t_one = time.perf_counter() - t1
    finally:
        oracle.set_num_threads(cores)
    return {"value": spec.npts / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "1 TVD-RK3 step of the 81^4 WENO5 x-subsystem from the cold start "
                      "(%.1f s)" % t,
            "one_core": {"value": small.npts / t_one, "unit": UNIT, "cores": 1,
                         "sample": "1 TVD-RK3 step of the 41^4 grid (%.1f s)" % t_one}}


def secondary_c1(hj, wl, stream, steps, peaks, peak_info):
    """The 41^4 cold solve + warm update pair from the b = 0 fixed point."""
    import numpy as np
    import torch
    spec = wl.config1(N_C1, BOUND_C1_PRIOR)
    g = hj.Grid.from_spec(spec, stream=stream)
    cap = dict(scheme=5, max_steps=200000, max_wall_ms=120000.0, band=BAND, band_margin=MARGIN,
               clamp=CLAMP)
    st = g.solve(hj.HJ_COLD, **cap)
    assert st["converged"], st
    prior = torch.empty(spec.npts, dtype=torch.float32, device="cuda")
    g.value_into(prior)
    g.set_disturbance_bound([-BOUND_C1], [BOUND_C1])
    hj.hj_jit_wait()

    def step():
        c = g.solve(hj.HJ_COLD, **cap)
        g.set_value(prior)
        w = g.solve(hj.HJ_WARM, **cap)
        return c, w

    step()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    t, updates, cold_ms, warm_ms, cs, wsteps = 0.0, 0, [], [], [], []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c, w = step()
        e1.record(stream)
        e1.synchronize()
        t += e0.elapsed_time(e1) / 1e3
        updates += spec.npts * (c["steps"] + w["steps"])
        cold_ms.append(c["wall_ms"])
        warm_ms.append(w["wall_ms"])
        cs.append(c["steps"])
        wsteps.append(w["steps"])
    Wc = torch.empty_like(prior)
    c = g.solve(hj.HJ_COLD, **cap)
    g.value_into(Wc)
    g.set_value(prior)
    g.solve(hj.HJ_WARM, **cap)
    Ww = torch.empty_like(prior)
    g.value_into(Ww)
    from paper_2101_05916_gb300 import scenarios
    acc = scenarios._acc(Ww.reshape(spec.n), Wc.reshape(spec.n), spec)
    per = stage_launch_seconds(hj, g, stream)
    peak, sms, mhz = peak_info
    roof = roofline_entry(hj, spec.npts, per, peak, sms, mhz, STAGE_TRAFFIC_BYTES_41,
                          kernel_name(hj, N_C1), peaks)
    g.close()
    return {"workload": "x4_41^4_weno5_cold+warm_update", "value": updates / t, "unit": UNIT,
            "steps": steps, "ms_per_step": 1e3 * t / steps,
            "cold_ms_p50": float(np.percentile(cold_ms, 50)),
            "warm_update_ms_p50": float(np.percentile(warm_ms, 50)),
            "cold_steps": int(np.median(cs)), "warm_steps": int(np.median(wsteps)),
            "warm_vs_cold_accuracy": acc, "roofline": roof}


def profile_only(args, hj, wl):
    """A few fixed TVD-RK3 steps on one 4-D grid, for ncu: the shape-specialised
    kernels are compiled and awaited first, so the profiled launches are the
    ones the bench times."""
    import torch
    spec = wl.quad_x4(args.profile_n, BOUND)
    g = hj.Grid.from_spec(spec, stream=torch.cuda.current_stream())
    if args.profile_tile:
        g.set_launch_shape(256, args.profile_tile)
    g.solve(hj.HJ_COLD, scheme=5, fixed_steps=1, clamp=CLAMP)
    hj.hj_jit_wait()
    st = g.solve(hj.HJ_COLD, scheme=5, fixed_steps=args.profile_steps, clamp=CLAMP)
    torch.cuda.synchronize()
    print(json.dumps({"profile_steps": st["steps"], "dt": st["dt"], "n": args.profile_n,
                      "launch_shape": g.launch_shape()}))
    g.close()


def main():
    t_start = time.perf_counter()
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    ws, rank, local = dist_setup(args)
    import numpy as np
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    from paper_2101_05916_gb300 import build as build_mod
    if rank == 0 or ws == 1:
        build_mod.build()
    barrier(ws)
    from paper_2101_05916_gb300 import hj
    from paper_2101_05916_gb300 import scenarios
    from paper_2101_05916_gb300 import workloads as wl

    if args.profile_steps:
        profile_only(args, hj, wl)
        return
    peaks = measured_peaks()
    peak_info = fp32_peak_tflops(peaks)
    stream = torch.cuda.current_stream()
    cs, fs = wl.quad_x4(N_COARSE, BOUND), wl.quad_x4(N_FINE, BOUND)
    gc = hj.Grid.from_spec(cs, stream=stream)
    gf = hj.Grid.from_spec(fs, stream=stream)
    opts = dict(scenarios.X4_OPTS, max_wall_ms=args.max_wall_ms)
    if args.no_graph:
        opts["use_graph"] = False

    def step():
        c = gc.solve(hj.HJ_COLD, **opts)
        hj.prolong(gc, gf)
        f = gf.solve(hj.HJ_WARM, **opts)
        return c, f

    # start the background compiles of the shape-specialised kernels of both
    # grids and wait for them, so that every warm-up and timed step uses them
    gc.solve(hj.HJ_COLD, scheme=5, fixed_steps=1, clamp=CLAMP)
    gf.solve(hj.HJ_COLD, scheme=5, fixed_steps=1, clamp=CLAMP)
    hj.hj_jit_wait()
    for _ in range(args.warmup):
        step()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    barrier(ws)

    sampler = ClockSampler(local)
    sampler.start()
    launches0 = hj.hj_kernel_launches()
    times, updates, lat_ms, c_steps, f_steps = [], 0, [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c, f = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        updates += cs.npts * c["steps"] + fs.npts * f["steps"]
        lat_ms.append(c["wall_ms"] + f["wall_ms"])
        c_steps.append(c["steps"])
        f_steps.append(f["steps"])
        assert c["converged"] and f["converged"], (c, f)
    torch.cuda.synchronize()
    launches = hj.hj_kernel_launches() - launches0
    clocks = sampler.stop()
    barrier(ws)
    t_local = sum(times)
    t_max = reduce_max(ws, t_local)
    total_updates = reduce_sum(ws, float(updates))
    value = total_updates / t_max

    if args.only_headline:
        gc.close()
        gf.close()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                              "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": 1e3 * t_max / args.steps,
                              "config": arm_config(), "gpu_launches": int(launches),
                              "clocks": clocks, "only_headline": True}))
        return

    # ---- accuracy of the update against the plain cold fine solve, and its latency
    W_upd = torch.empty(fs.npts, dtype=torch.float32, device="cuda")
    gf.value_into(W_upd)
    torch.cuda.synchronize()
    cold = gf.solve(hj.HJ_COLD, **opts)
    W_cold = torch.empty_like(W_upd)
    gf.value_into(W_cold)
    acc = scenarios._acc(W_upd.reshape(fs.n), W_cold.reshape(fs.n), fs)
    ref = scenarios.load_reference(os.path.join(ROOT, "tests", "golden",
                                                "x41_b1.0_monotone_band_samples.txt"))
    vs_oracle = None
    if ref is not None:
        idx = torch.as_tensor(ref["idx"] * 2, device="cuda")
        Wn = W_upd.reshape(fs.n)[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]].double().cpu().numpy()
        vs_oracle = {"max_abs": float(np.abs(Wn - ref["W"]).max()),
                     "sign_agreement": float(np.mean((Wn >= 0) == (ref["W"] >= 0))),
                     "note": "81^4 update restricted to every second node vs the FP64 "
                             "oracle's converged 41^4 solve (a discretisation report)"}

    # ---- roofline of the dominant kernel: the WENO5 stage on the 81^4 grid
    per_launch = stage_launch_seconds(hj, gf, stream)
    peak, sms, mhz = peak_info
    roofline = roofline_entry(hj, fs.npts, per_launch, peak, sms, mhz, STAGE_TRAFFIC_BYTES_81,
                              kernel_name(hj, N_FINE), peaks)
    fine_launches = 3 * sum(f_steps)
    roofline["fine_stage_share_of_timed_region"] = per_launch * fine_launches / t_local
    gc.close()
    gf.close()

    # ---- end to end through the C ABI from a host description of the problem
    e2e = None
    if not args.no_e2e:
        out_host = torch.empty(fs.npts, dtype=torch.float32, pin_memory=True)
        e2e_t, e2e_updates, h2d = 0.0, 0, 0
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            a = hj.Grid.from_spec(cs, stream=stream)
            b = hj.Grid.from_spec(fs, stream=stream)
            c = a.solve(hj.HJ_COLD, **opts)
            hj.prolong(a, b)
            f = b.solve(hj.HJ_WARM, **opts)
            b.value_into(out_host)           # D2H: the updated fine value function
            a.close()
            b.close()
            e1.record(stream)
            e1.synchronize()
            e2e_t += e0.elapsed_time(e1) / 1e3
            e2e_updates += cs.npts * c["steps"] + fs.npts * f["steps"]
        # host inputs per step: the two problem descriptions passed by value
        # (axis counts, box, model parameters, wind interval, constraint box)
        for sp in (cs, fs):
            h2d += 4 * sp.ndim + 8 * (2 * sp.ndim + len(sp.params) + 2 * len(sp.d_lo)
                                      + 2 * sp.ndim)
        e2e_t = reduce_max(ws, e2e_t)
        e2e = {"value": reduce_sum(ws, float(e2e_updates)) / e2e_t, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4 * fs.npts,
               "note": "grids created from the host description, solved, value read back "
                       "into pinned host memory and destroyed inside every step"}

    secondary = secondary_c1(hj, wl, stream, args.secondary_steps, peaks, peak_info)

    # ---- scenarios: the paper's accelerations against the plain cold way
    scen = None
    if not args.no_scenarios:
        scen = {"decomposed_update": scenarios.decomposed_update(),
                "adaptive_grid": scenarios.adaptive_grid(reference=ref),
                "local_wind_update": scenarios.local_wind_update(),
                "localized_update": scenarios.localized_update(),
                "moving_constraint": scenarios.moving_constraint(),
                "safety_filter": scenarios.safety_filter(),
                "serving": scenarios.serving(
                    args.serve_requests,
                    forms=("served", "served_coarse_init") if args.serve_coarse else ("served",))}
    if rank != 0:
        return
    latency = {
        "adaptive_update_p50": float(np.percentile(lat_ms, 50)),
        "adaptive_update_p99": float(np.percentile(lat_ms, 99)),
        "plain_cold_81^4": float(cold["wall_ms"]),
        "plain_cold_81^4_steps": int(cold["steps"]),
        "adaptive_coarse_steps": int(np.median(c_steps)),
        "adaptive_fine_steps": int(np.median(f_steps)),
        "adaptive_vs_cold_accuracy": acc,
        "adaptive_meets_bar": acc["meets_bar"],
    }
    if scen is not None:
        sv = scen["serving"]
        latency["serving_requests"] = sv["requests"]
        latency["plain_cold_p50"] = sv["plain_cold"]["p50_ms"]
        latency["plain_cold_p99"] = sv["plain_cold"]["p99_ms"]
        for f in ("served", "served_coarse_init"):
            if f not in sv:
                continue
            if sv[f]["accuracy"]["meets_bar"]:
                latency[f + "_p50"] = sv[f]["p50_ms"]
                latency[f + "_p99"] = sv[f]["p99_ms"]
            else:
                latency[f] = "below the bar (%d of %d requests at it)" % (
                    sv[f]["accuracy"]["requests_meeting_bar"], sv[f]["accuracy"]["requests"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": arm_config(),
        "latency_ms": latency,
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "vs_oracle_41": vs_oracle,
        "secondary": secondary,
    }
    if scen is not None:
        line["scenarios"] = scen
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    line["bench_wall_s"] = time.perf_counter() - t_start
    print(json.dumps(line))


if __name__ == "__main__":
    main()
