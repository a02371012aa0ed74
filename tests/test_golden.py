"""Stored oracle outputs and the paper's printed constants.

The .txt fixtures were written by tests/golden/make_golden.py, which calls only
the oracle; they guard the oracle against unintended changes.  The constants
fixture holds numbers printed in the paper with their section, and checks that
the workload definitions use them.
"""
import json
import os

import numpy as np

import oracle
from paper_2101_05916_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


def test_oracle_matches_stored_z41():
    s = wl.quad_z(41, 0.5)
    W, st = oracle.solve(s, scheme=2, tol=1e-9, max_steps=50000)
    ref = _load("z41_eno2_b0.5_converged.txt").reshape(s.n)
    assert np.abs(W - ref).max() < 1e-12


def test_oracle_matches_stored_x9():
    x = wl.quad_x4(9, 0.5)
    W, st = oracle.solve(x, scheme=5, fixed_steps=5)
    ref = _load("x9_weno5_b0.5_5steps.txt").reshape(x.n)
    assert np.abs(W - ref).max() < 1e-12


def test_workload_constants_follow_the_paper():
    c = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    g, d1, d0, n0 = wl.X4_PARAMS[:4]
    assert d0 == c["quad10d_d0"]["value"]
    assert d1 == c["quad10d_d1"]["value"]
    assert n0 == c["quad10d_n0"]["value"]


def test_serving_trace_matches_the_committed_trace():
    """The seeded serving trace (the serving workload) is the one committed
    under tests/golden/ (written by make_serving_trace.py)."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    import make_serving_trace
    stored = json.load(open(os.path.join(here, "serving_trace_c4.json")))["requests"]
    assert make_serving_trace.trace_records() == stored
    assert len(stored) == 256 and stored[-1]["arrival_s"] > 10.0
