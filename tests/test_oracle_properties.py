"""Randomised pins of the oracle (Hypothesis; skipped where it is absent).

With dx/dt = d, |d| <= b and no control, every point of [x - b s, x + b s]
is reachable, so for any constraint l the value after time s is the minimum
of l over that window.  For random piecewise-linear safe sets (convex or
not) the oracle's ENO2 and WENO5 solves must match that window minimum:
to rounding away from its kinks (the schemes are exact on linear pieces),
and at them within a few cells times the slopes of l.
"""
import numpy as np
import pytest

import oracle
from paper_2101_05916_gb300 import workloads as wl

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies


@hypothesis.settings(max_examples=30, deadline=None,
                     suppress_health_check=[hypothesis.HealthCheck.too_slow])
@hypothesis.given(n=st.integers(81, 161), b=st.floats(0.1, 0.8), T=st.floats(0.1, 0.6),
                  pts=st.lists(st.tuples(st.floats(-2.4, 2.4), st.floats(-0.6, 0.6)),
                               min_size=2, max_size=5, unique_by=lambda p: round(p[0], 2)),
                  scheme=st.sampled_from([2, 5]))
def test_drift_value_is_the_window_minimum_of_any_constraint(n, b, T, pts, scheme):
    s = wl.drift((n,), 2.5, b, wl.CON_BOX, r=1.0)
    x = s.coords()[0]
    h = s.h()[0]
    pts = sorted(pts)
    px = np.array([p[0] for p in pts])
    py = np.array([p[1] for p in pts])

    def l_of(y):
        return np.interp(y, np.concatenate([[-10.0], px, [10.0]]),
                         np.concatenate([[py[0]], py, [py[-1]]]))

    W, _ = oracle.solve(s, scheme=scheme, dt=T / 100, fixed_steps=100, lfield=l_of(x))
    ys = np.linspace(-b * T, b * T, 2001)
    exact = np.array([l_of(xi + ys).min() for xi in x])
    # away from the faces, where the window would leave the grid
    inner = np.abs(x) < 2.5 - (b * T + 6 * h)
    hypothesis.assume(inner.sum() > 10)
    err = np.abs(W - exact)[inner]
    # the schemes smooth a kink over a few cells: the error there scales
    # with the slopes of l
    lip = max(1.0, float(np.max(np.abs(np.diff(py) / np.maximum(np.diff(px), 1e-9))))
              if len(px) > 1 else 1.0)
    assert err.mean() < 0.35 * h * lip
    assert err.max() < 10.0 * h * lip
    # the window minimum's kinks: l's breakpoints and those moved by +-b s
    kinks = np.concatenate([px, px - b * T, px + b * T])
    far = inner & (np.abs(x[:, None] - kinks[None, :]).min(axis=1) > 14 * h)
    if far.any():
        assert np.abs(W - exact)[far].max() < 1e-5 * h
    # W <= l and the value never rises above its start (no control, VI clamp)
    assert np.all(W <= l_of(x) + 1e-12)
