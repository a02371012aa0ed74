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


def _box_margin(lo, hi):
    def l_of(x, y):
        inside = (x >= lo[0]) & (x <= hi[0]) & (y >= lo[1]) & (y <= hi[1])
        m = np.minimum(np.minimum(x - lo[0], hi[0] - x), np.minimum(y - lo[1], hi[1] - y))
        ex = np.maximum(np.maximum(lo[0] - x, x - hi[0]), 0.0)
        ey = np.maximum(np.maximum(lo[1] - y, y - hi[1]), 0.0)
        return np.where(inside, m, -np.hypot(ex, ey))
    return l_of


def _drift2_error(n, lo, hi, dlo, dhi, T):
    """Mean |W - exact| over interior nodes for a 2-D drift with the
    disturbance box [dlo, dhi] (asymmetric, possibly excluding 0) and the
    box constraint [lo, hi]: every point t v, t in [0, T], v in the box, is
    reachable, so W(x) is the minimum of l over x + that cone."""
    import dataclasses
    s = wl.drift((n, n), 2.0, 0.3, wl.CON_BOX, r=1.0)
    s = dataclasses.replace(s, d_lo=tuple(dlo), d_hi=tuple(dhi), con_a=tuple(lo),
                            con_b=tuple(hi))
    h = s.h()[0]
    steps = int(np.ceil(T / min(T / 120, 0.25 * h / max(np.abs(np.r_[dlo, dhi]).max(), 1e-9))))
    W, _ = oracle.solve(s, scheme=2, dt=T / steps, fixed_steps=steps)
    xs = s.coords()
    l_of = _box_margin(lo, hi)
    a = np.linspace(0.0, 1.0, 17)
    A1, A2, TT = np.meshgrid(a, a, np.linspace(0.0, T, 17), indexing="ij")
    ox = (TT * (dlo[0] + A1 * (dhi[0] - dlo[0]))).ravel()
    oy = (TT * (dlo[1] + A2 * (dhi[1] - dlo[1]))).ravel()
    exact = np.array([[l_of(x + ox, y + oy).min() for y in xs[1]] for x in xs[0]])
    X, Y = np.meshgrid(*xs, indexing="ij")
    reach = np.abs(np.r_[dlo, dhi]).max() * T
    inner = (np.abs(X) < 2.0 - reach - 0.3) & (np.abs(Y) < 2.0 - reach - 0.3)
    return float(np.abs(W - exact)[inner].mean()), h


@pytest.mark.parametrize("seed", [0, 3, 4])
def test_drift2_asymmetric_disturbance_converges_to_the_reachable_minimum(seed):
    """2-D, asymmetric disturbance intervals (Sec. II-C: a GP interval need
    not be centred), random box: the ENO2 oracle converges to the exact
    value under refinement.  A wrong sign, a swapped bound or a dropped
    axis in H leaves an O(1) error that does not shrink."""
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-1.3, -0.3, 2)
    hi = rng.uniform(0.3, 1.3, 2)
    dlo = rng.uniform(-0.6, 0.3, 2)
    dhi = dlo + rng.uniform(0.0, 0.6, 2)
    T = float(rng.uniform(0.2, 0.8))
    e41, h41 = _drift2_error(41, lo, hi, dlo, dhi, T)
    e81, _ = _drift2_error(81, lo, hi, dlo, dhi, T)
    assert e41 < 0.1 * h41
    assert e81 < 0.6 * e41
