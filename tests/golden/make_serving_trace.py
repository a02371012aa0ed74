"""Writes serving_trace_c4.json: the 256-request serving trace (Poisson
arrivals at 20/s, seed 20210115, PCG64) as generated by
workloads.serving_trace, so that a change of the generator or of NumPy's
random streams shows up as a test failure instead of a silently different
workload.  Holds inputs only."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2101_05916_gb300 import workloads as wl  # noqa: E402


def trace_records():
    out = []
    for r in wl.serving_trace():
        s = r.spec
        out.append({"rid": r.rid, "arrival_s": round(r.arrival_s, 9), "name": s.name,
                    "model": s.model, "n": list(s.n), "d_hi": [round(v, 12) for v in s.d_hi],
                    "con_a": [None if abs(v) == float("inf") else round(v, 12) for v in s.con_a],
                    "con_b": [None if abs(v) == float("inf") else round(v, 12) for v in s.con_b],
                    "scheme": r.scheme})
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "serving_trace_c4.json"), "w") as f:
        json.dump({"generator": "workloads.serving_trace(count=256, rate_hz=20, seed=20210115)",
                   "requests": trace_records()}, f, indent=0)
        f.write("\n")
