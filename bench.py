"""Benchmark: HJ grid-point updates/s of the safe-set solve on GB300.

Workload (default): the 4-D x-subsystem of the decomposed near-hover
quadcopter on a 41^4 grid, WENO5 + TVD-RK3, CFL 0.5, clamp min(W3, l, W_prev)
(the monotone tube), stop at an L-inf change below 1e-4 per 0.1 s window on
the band |W| <= 0.5 around the safe-set boundary, wind bound |d| <= 0.5.  One bench step is one
safe-set update pair:
    (1) a cold solve from the constraint margin, to convergence;
    (2) a warm-started update (Sec. III-B) from the device-resident fixed
        point of the previous bound (|d| <= 0), to convergence.
One grid-point update is one node advanced by one full TVD-RK3 step.
value = total updates / total device time of the K timed steps.  L2 is
flushed between timed steps (the 45 MB working set would otherwise stay
resident across steps).

Other lines: `e2e` repeats the step through the same C ABI with the prior
uploaded from pinned host memory and both results read back.
`latency_ms` gives p50/p99 of the cold solve and the warm update, and of the
served form vs one-at-a-time cold solves on the first requests of the seeded
serving trace.  `scenarios` holds the decomposed batched update (x, y at 61^4
and z at 201^2, wind 0 -> 0.5 -> 1.0 -> 1.5), the coarse-to-fine solve
(31^4 -> 81^4), and the serving sample.
`roofline` times the dominant stage kernel in a separate fixed-step pass with
CUDA events.  `cpu_baseline` is the FP64 oracle timed on a bounded sample of
the same workload.

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
N_AXIS = 41
BOUND_PRIOR, BOUND = 0.0, 0.5
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
# DRAM bytes per stage launch (read + write, average of stages 1-3) from the
# ncu capture summarised in profiles/stage_kernel_x41_weno5.md; set to None
# whenever the stage kernel changes until it is captured again.
STAGE_TRAFFIC_BYTES = (11.316736e6 + 22.620416e6 + 22.622720e6) / 3.0
# FP32 non-tensor peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


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
    ap.add_argument("--serve-requests", type=int, default=16)
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run only this many fixed TVD-RK3 steps of the workload (for ncu)")
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


# ------------------------------------------------------------- reference arm

def arm_config():
    """The workload both arms report: the 41^4 x subsystem, WENO5, TVD-RK3."""
    return {"workload": "x4_41^4_weno5_cold+warm_update", "grid": [N_AXIS] * 4,
            "scheme": "WENO5", "rk": "TVD-RK3", "cfl": 0.5, "tol": 1e-4,
            "check_dt": 0.1, "stop_band": BAND, "clamp": "monotone", "wind_prior": BOUND_PRIOR,
            "wind": BOUND, "l2": "flushed between timed steps",
            "parallelism": "independent grids per rank"}


def run_reference(args):
    """The FP64 oracle as the reference arm: each step advances a bounded
    sample (2 TVD-RK3 steps of the 41^4 WENO5 x-subsystem) on the host cores."""
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    from paper_2101_05916_gb300 import workloads as wl
    spec = wl.config1(N_AXIS, BOUND)
    dt = oracle.cfl_dt(spec)
    sample_steps = 2
    for _ in range(args.warmup):
        oracle.solve(spec, scheme=5, dt=dt, fixed_steps=1)
    t = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.solve(spec, scheme=5, dt=dt, fixed_steps=sample_steps)
        t += time.perf_counter() - t0
    updates = spec.npts * sample_steps * args.steps
    v = updates / t
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(arm_config(),
                       sample="%d TVD-RK3 steps of the same grid and scheme per bench step"
                              % sample_steps),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d RK3 steps of 41^4 WENO5 per step, %d steps"
                                   % (sample_steps, args.steps)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------- gb300 arm

def cpu_baseline():
    import oracle
    from paper_2101_05916_gb300 import workloads as wl
    spec = wl.config1(N_AXIS, BOUND)
    dt = oracle.cfl_dt(spec)
    oracle.solve(spec, scheme=5, dt=dt, fixed_steps=1)  # warm the pages
    k = 8
    t0 = time.perf_counter()
    oracle.solve(spec, scheme=5, dt=dt, fixed_steps=k)
    t = time.perf_counter() - t0
    return {"value": spec.npts * k / t, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "%d TVD-RK3 steps of the 41^4 WENO5 x-subsystem from the cold start "
                      "(%.1f s)" % (k, t)}


def main():
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
    from paper_2101_05916_gb300 import workloads as wl

    stream = torch.cuda.current_stream()
    spec = wl.config1(N_AXIS, BOUND_PRIOR)
    g = hj.Grid.from_spec(spec, stream=stream)
    npts = spec.npts
    # prior: converged value function of the previous (smaller) wind bound
    if args.profile_steps:
        g.set_disturbance_bound([-BOUND], [BOUND])
        # the shape-specialised kernels compile in the background: start and
        # wait for them, so that the profiled launches are the ones timed
        g.solve(hj.HJ_COLD, scheme=5, fixed_steps=1, clamp=CLAMP)
        hj.hj_jit_wait()
        st = g.solve(hj.HJ_COLD, scheme=5, fixed_steps=args.profile_steps, clamp=CLAMP)
        torch.cuda.synchronize()
        print(json.dumps({"profile_steps": st["steps"], "dt": st["dt"]}))
        g.close()
        return
    st_prior = g.solve(hj.HJ_COLD, scheme=5, max_steps=200000, max_wall_ms=120000.0, band=BAND,
                       band_margin=MARGIN, clamp=CLAMP)
    assert st_prior["converged"], st_prior
    prior = torch.empty(npts, dtype=torch.float32, device="cuda")
    g.value_into(prior)
    g.set_disturbance_bound([-BOUND], [BOUND])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    cap = dict(scheme=5, max_steps=200000, max_wall_ms=120000.0, band=BAND, band_margin=MARGIN,
               clamp=CLAMP)

    def step():
        c = g.solve(hj.HJ_COLD, **cap)
        g.set_value(prior)
        w = g.solve(hj.HJ_WARM, **cap)
        return c, w

    # the prior's solve started the background compile of the shape-specialised
    # kernels; the warm-up steps run with them
    hj.hj_jit_wait()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)

    sampler = ClockSampler(local)
    sampler.start()
    launches0 = hj.hj_kernel_launches()
    times, updates, cold_ms, warm_ms, cold_steps, warm_steps = [], 0, [], [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c, w = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        updates += npts * (c["steps"] + w["steps"])
        cold_ms.append(c["wall_ms"])
        warm_ms.append(w["wall_ms"])
        cold_steps.append(c["steps"])
        warm_steps.append(w["steps"])
        assert c["converged"] and w["converged"], (c, w)
    torch.cuda.synchronize()
    launches = hj.hj_kernel_launches() - launches0
    clocks = sampler.stop()
    barrier(ws)
    t_local = sum(times)
    t_max = reduce_max(ws, t_local)
    total_updates = reduce_sum(ws, float(updates))
    value = total_updates / t_max

    # ---- roofline of the dominant kernel: WENO5 4-D stage, fixed-step pass
    kpass = 60
    g.set_value(prior)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.solve(hj.HJ_WARM, scheme=5, fixed_steps=kpass, clamp=CLAMP)
    e1.record(stream)
    e1.synchronize()
    per_launch_s = e0.elapsed_time(e1) / 1e3 / (3 * kpass)
    flops_launch = FLOPS_PER_UPDATE[("quad_x4", 5)] / 3.0 * npts
    achieved_tflops = flops_launch / per_launch_s / 1e12
    hbm_gbs = BYTES_PER_UPDATE / 3.0 * npts / per_launch_s / 1e9
    peaks = measured_peaks()
    roofline = {
        "bound": "alu",
        "kernel": ("hj_stage_1..3 (stage kernel, WENO5, quad_x4, specialised to the 41^4 shape)"
                   if hj.hj_jit_kernels() > 0 else "stage_kernel<4,WENO5,quad_x4>"),
        "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": achieved_tflops / FP32_PEAK_TFLOPS,
        "peak_source": "FP32 lanes x max SM clock (152 x 128 x 2 x 2.07 GHz)",
        "per_launch_us": per_launch_s * 1e6,
        "flops_per_update": FLOPS_PER_UPDATE[("quad_x4", 5)],
        "traffic": STAGE_TRAFFIC_BYTES,
        "algorithmic_bytes_per_launch": BYTES_PER_UPDATE / 3.0 * npts,
        "hbm_view": {"achieved_gbs": hbm_gbs, "bytes_per_update": BYTES_PER_UPDATE,
                     "peak_gbs": peaks["hbm_gbs"] if peaks else 6800.0,
                     "frac": hbm_gbs / (peaks["hbm_gbs"] if peaks else 6800.0),
                     "peak_source": "measured" if peaks else "fallback"},
    }

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        prior_host = torch.empty(npts, dtype=torch.float32, pin_memory=True)
        prior_host.copy_(prior.cpu())
        out_host = torch.empty(npts, dtype=torch.float32, pin_memory=True)
        e2e_t, e2e_updates = 0.0, 0
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c = g.solve(hj.HJ_COLD, **cap)
            g.value_into(out_host)           # D2H: cold result
            g.set_value(prior_host)          # H2D: prior from the host
            w = g.solve(hj.HJ_WARM, **cap)
            g.value_into(out_host)           # D2H: updated value function
            e1.record(stream)
            e1.synchronize()
            e2e_t += e0.elapsed_time(e1) / 1e3
            e2e_updates += npts * (c["steps"] + w["steps"])
        e2e_t = reduce_max(ws, e2e_t)
        e2e = {"value": reduce_sum(ws, float(e2e_updates)) / e2e_t, "unit": UNIT,
               "h2d_bytes_per_step": 4 * npts, "d2h_bytes_per_step": 8 * npts}

    g.close()

    # ---- scenarios: the paper's accelerations against the plain cold way
    scen = None
    if not args.no_scenarios:
        from paper_2101_05916_gb300 import scenarios
        ref = scenarios.load_reference(os.path.join(ROOT, "tests", "golden",
                                                    "x41_b1.0_monotone_band_samples.txt"))
        scen = {"decomposed_update": scenarios.decomposed_update(),
                "adaptive_grid": scenarios.adaptive_grid(reference=ref),
                "local_wind_update": scenarios.local_wind_update(),
                "moving_constraint": scenarios.moving_constraint(),
                "safety_filter": scenarios.safety_filter(),
                "serving": scenarios.serving(args.serve_requests)}
    if rank != 0:
        return
    latency = {
        "x41_cold_p50": float(np.percentile(cold_ms, 50)),
        "x41_cold_p99": float(np.percentile(cold_ms, 99)),
        "x41_warm_update_p50": float(np.percentile(warm_ms, 50)),
        "x41_warm_update_p99": float(np.percentile(warm_ms, 99)),
        "x41_cold_steps": int(np.median(cold_steps)), "x41_warm_steps": int(np.median(warm_steps))}
    if scen is not None:
        sv = scen["serving"]
        latency.update({"served_p50": sv["served"]["p50_ms"], "served_p99": sv["served"]["p99_ms"],
                        "served_coarse_init_p50": sv["served_coarse_init"]["p50_ms"],
                        "served_coarse_init_p99": sv["served_coarse_init"]["p99_ms"],
                        "served_coarse_init_eno2_p50": sv["served_coarse_init_eno2"]["p50_ms"],
                        "served_coarse_init_eno2_p99": sv["served_coarse_init_eno2"]["p99_ms"],
                        "plain_cold_p50": sv["plain_cold"]["p50_ms"],
                        "plain_cold_p99": sv["plain_cold"]["p99_ms"],
                        "serving_requests": sv["requests"]})
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
    }
    if scen is not None:
        line["scenarios"] = scen
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
