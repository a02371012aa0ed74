"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against a closed form, a textbook property, an
invariant of the HJI variational inequality (Eq. 2), or an independent
brute-force solution of the differential game behind Eq. 1.  A dropped term,
a flipped sign, or a wrong index anywhere in the oracle fails at least one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2101_05916_gb300 import workloads as wl

pytestmark = pytest.mark.filterwarnings("ignore")


# ------------------------------------------------------------ one-sided slopes

@pytest.mark.parametrize("scheme,deg", [(1, 1), (2, 2), (5, 3)])
def test_slopes_exact_on_polynomials(scheme, deg):
    """Every candidate stencil is exact on polynomials of its degree, so the
    scheme is exact whatever its nonlinear weights (Osher & Fedkiw 3.3-3.4)."""
    rng = np.random.default_rng(7)
    n, h = 40, 0.1
    x = -1.3 + h * np.arange(n)
    for _ in range(5):
        c = rng.standard_normal(deg + 1)
        w = np.polyval(c, x)
        dw = np.polyval(np.polyder(c), x)
        pm, pp = oracle.line_slopes(w, h, scheme)
        r = {1: 1, 2: 2, 5: 3}[scheme]
        sl = slice(r, n - r)
        scale = np.abs(dw).max() + 1.0
        assert np.abs(pm[sl] - dw[sl]).max() < 1e-9 * scale
        assert np.abs(pp[sl] - dw[sl]).max() < 1e-9 * scale


@pytest.mark.parametrize("scheme", [1, 2, 5])
def test_slopes_exact_on_lines_including_ghosts(scheme):
    """Linear ghost extrapolation reproduces an affine line exactly at every node."""
    x = np.linspace(-2.0, 3.0, 17)
    w = 0.7 * x - 1.1
    pm, pp = oracle.line_slopes(w, x[1] - x[0], scheme)
    assert np.allclose(pm, 0.7, atol=1e-12) and np.allclose(pp, 0.7, atol=1e-12)


@pytest.mark.parametrize("scheme,order", [(1, 0.9), (2, 1.8), (5, 4.5)])
def test_slopes_convergence_order(scheme, order):
    """On a smooth function the error falls as h^k: first-order 1, ENO2 2,
    WENO5 5 (the latter only with the right linear weights 1/10, 6/10, 3/10)."""
    errs = []
    for n in (41, 81):
        x = np.linspace(0.0, 1.0, n)
        h = x[1] - x[0]
        w = np.sin(2.0 * x) + 0.3 * np.cos(5.0 * x)
        dw = 2.0 * np.cos(2.0 * x) - 1.5 * np.sin(5.0 * x)
        pm, pp = oracle.line_slopes(w, h, scheme)
        mid = (x > 0.3) & (x < 0.7)
        errs.append(max(np.abs(pm - dw)[mid].max(), np.abs(pp - dw)[mid].max()))
    rate = math.log2(errs[0] / errs[1])
    assert rate > order, (errs, rate)


def test_weno5_is_non_oscillatory_at_a_jump():
    """The smoothness indicators must switch off stencils that cross a jump:
    left of the jump the left-biased slope stays at the (zero) slope of the
    smooth side, not the O(1/h) slope of the jump."""
    h = 0.1
    w = np.where(np.arange(30) < 15, 0.0, 1.0)
    pm, pp = oracle.line_slopes(w, h, 5)
    # node 13: the left-biased stencils {10..13}, {11..14} are smooth, {12..15} is not
    assert abs(pm[13]) < 1e-3
    assert abs(pp[11]) < 1e-3
    pm2, _ = oracle.line_slopes(w, h, 2)
    assert abs(pm2[13]) < 1e-12


# ---------------------------------------------------------------- constraint

def test_box_margin_values():
    s = wl.quad_x4(5, 0.0, 4.0)
    assert oracle.margin_at(s, [1.0, 0, 0, 0]) == pytest.approx(3.0)
    assert oracle.margin_at(s, [-3.5, 0, 0, 0]) == pytest.approx(0.5)
    assert oracle.margin_at(s, [4.5, 1.9, 0.3, -1.4]) == pytest.approx(-0.5)
    b = wl.drift((5, 5), 2.0, 0.1, wl.CON_BOX, r=1.0)
    assert oracle.margin_at(b, [2.0, 2.0]) == pytest.approx(-math.sqrt(2.0))
    assert oracle.margin_at(b, [0.5, -0.25]) == pytest.approx(0.5)
    o = wl.drift((5, 5), 2.0, 0.1, wl.CON_BALL_OUT, r=1.0)
    assert oracle.margin_at(o, [0.6, 0.8]) == pytest.approx(0.0)
    assert oracle.margin_at(o, [0.0, 0.0]) == pytest.approx(-1.0)


# ----------------------------------------------------------- dissipation, dt

def test_alpha_and_dt_closed_form_x4():
    """a_i = max |f_i| over the grid box and input box, in closed form for the
    4-D subsystem, and dt = 0.5 / sum a_i / h_i."""
    s = wl.config1()
    a = oracle.alpha(s)
    expect = [2.0 + 0.5, 9.81 * math.tan(0.35), 8.0 * 0.35 + 1.5,
              10.0 * 0.35 + 10.0 * math.pi / 9.0]
    assert np.allclose(a, expect, rtol=1e-12)
    h = s.h()
    assert oracle.cfl_dt(s) == pytest.approx(0.5 / sum(e / hh for e, hh in zip(expect, h)))
    assert oracle.cfl_dt(s) == pytest.approx(1.2996e-3, rel=1e-3)


def test_alpha_closed_form_z():
    s = wl.quad_z(101, 0.5)
    a = oracle.alpha(s)
    assert np.allclose(a, [3.0, max(abs(0.91 * 19.62 - 9.81) + 0.5, 9.81 + 0.5)])


def test_hamiltonian_max_min_order():
    """max_u min_d differs from min_d max_u only when u and d interact; here
    they enter additively, and H at hand-picked points has a closed value."""
    s = wl.quad_z(11, 0.5)
    # p = (0, 1): control pushes up at full thrust, wind pushes down
    assert oracle.hamiltonian(s, [1.0, 0.0], [0.0, 1.0]) == pytest.approx(
        0.91 * 19.62 - 9.81 - 0.5)
    # p = (0, -1): control cuts thrust, wind pushes up
    assert oracle.hamiltonian(s, [1.0, 0.0], [0.0, -1.0]) == pytest.approx(9.81 - 0.5)
    # p = (1, 0): no input acts, H = vz
    assert oracle.hamiltonian(s, [1.0, -1.7], [1.0, 0.0]) == pytest.approx(-1.7)
    x = wl.quad_x4(5, 0.5)
    # p on the disturbed axis only: H = p1 v - b |p1|
    assert oracle.hamiltonian(x, [0, 1.0, 0, 0], [2.0, 0, 0, 0]) == pytest.approx(2.0 - 1.0)
    # p on the controlled axis only: H = p4 (-d0 th) + n0 umax |p4|
    assert oracle.hamiltonian(x, [0, 0, 0.1, 0], [0, 0, 0, -1.0]) == pytest.approx(
        1.0 + 10.0 * math.pi / 9.0)


def test_hamiltonian_asymmetric_input_boxes_x4():
    """x subsystem with asymmetric control and disturbance boxes: the sign
    with which u enters dw/dt decides H (with a symmetric box it would not).
    H = p0 v + p1 g tan(th) + p2 (-d1 th + w) + p3 (-d0 th)
        + max_u p3 n0 u + min_d p0 d."""
    import dataclasses
    x = dataclasses.replace(wl.quad_x4(5, 0.5), params=(9.81, 8.0, 10.0, 10.0, -0.1, 0.3, 0.0),
                            d_lo=(-0.2,), d_hi=(0.6,))
    st = [0.0, 0.0, 0.2, 0.0]
    assert oracle.hamiltonian(x, st, [0, 0, 0, 1.0]) == pytest.approx(-2.0 + 10.0 * 0.3)
    assert oracle.hamiltonian(x, st, [0, 0, 0, -1.0]) == pytest.approx(2.0 + 10.0 * 0.1)
    # disturbance on dx/dt: min over [-0.2, 0.6] of p0 d
    st2 = [0.0, 0.5, 0.0, 0.0]
    assert oracle.hamiltonian(x, st2, [1.0, 0, 0, 0]) == pytest.approx(0.5 - 0.2)
    assert oracle.hamiltonian(x, st2, [-1.0, 0, 0, 0]) == pytest.approx(-0.5 - 0.6)


# ------------------------------------------------------------- closed forms

@pytest.mark.parametrize("scheme", [2, 5])
def test_drift_1d_ball_exterior(scheme):
    """dx/dt = d, |d| <= b, safe |x| >= r:  W(x, s) = max(|x| - b s, 0) - r."""
    b, r, T = 0.5, 0.3, 0.6
    s = wl.drift((201,), 2.0, b, wl.CON_BALL_OUT, r=r)
    W, st = oracle.solve(s, scheme=scheme, dt=T / 60, fixed_steps=60)
    x = s.coords()[0]
    exact = np.maximum(np.abs(x) - b * T, 0.0) - r
    h = s.h()[0]
    interior = slice(4, -4)
    assert np.abs(W - exact)[interior].max() < 1.5 * h
    # outside the eroded front the value is affine, where every scheme is exact
    # (inside it, WENO5 keeps an O(h) undershoot from the initial kink of l)
    away = np.abs(x) > b * T + 10 * h
    assert np.abs(W - exact)[away].max() < 1e-6
    assert np.all(W <= oracle.margin(s) + 1e-15)


@pytest.mark.parametrize("scheme", [2, 5])
def test_drift_1d_box(scheme):
    """Safe inside |x| <= r: the disturbance erodes the margin at rate b."""
    b, r, T = 0.8, 1.5, 0.5
    s = wl.drift((101,), 2.0, b, wl.CON_BOX, r=r)
    W, _ = oracle.solve(s, scheme=scheme, dt=T / 50, fixed_steps=50)
    x = s.coords()[0]
    exact = r - b * T - np.abs(x)
    away = np.abs(x) > 3 * s.h()[0]
    assert np.abs(W - exact)[away].max() < 1e-9


@pytest.mark.parametrize("ndim", [2, 3])
def test_drift_nd_ball_exterior_box_disturbance(ndim):
    """Box disturbance |d_i| <= b:  W = || max(|x_i| - b s, 0) || - r."""
    b, r, T = 0.4, 0.5, 0.5
    n = 41 if ndim == 2 else 25
    s = wl.drift((n,) * ndim, 2.0, b, wl.CON_BALL_OUT, r=r)
    W, _ = oracle.solve(s, scheme=5, dt=T / 40, fixed_steps=40)
    X = np.meshgrid(*s.coords(), indexing="ij")
    exact = np.sqrt(sum(np.maximum(np.abs(xi) - b * T, 0.0) ** 2 for xi in X)) - r
    h = s.h()[0]
    inner = tuple(slice(3, -3) for _ in range(ndim))
    assert np.abs(W - exact)[inner].max() < 2.0 * h
    assert np.abs(W - exact)[inner].mean() < 0.1 * h


@pytest.mark.parametrize("ndim", [2, 3])
def test_drift_nd_box_constraint(ndim):
    """Box constraint and box disturbance: W is the margin to the box shrunk by b s."""
    b, r, T = 0.4, 1.2, 0.5
    n = 41 if ndim == 2 else 25
    s = wl.drift((n,) * ndim, 2.0, b, wl.CON_BOX, r=r)
    W, _ = oracle.solve(s, scheme=5, dt=T / 40, fixed_steps=40)
    shrunk = wl.drift((n,) * ndim, 2.0, b, wl.CON_BOX, r=r - b * T)
    exact = oracle.margin(shrunk)
    h = s.h()[0]
    inner = tuple(slice(3, -3) for _ in range(ndim))
    assert np.abs(W - exact)[inner].max() < 2.0 * h
    assert np.abs(W - exact)[inner].mean() < 0.1 * h


@pytest.mark.parametrize("b", [0.5, 2.0])
@pytest.mark.parametrize("scheme", [2, 5])
def test_z_double_integrator_converged(b, scheme):
    """Converged z value = distance to the nearer wall after braking at full
    authority against the worst wind (bang-bang switching curves)."""
    errs = []
    for n in (101, 201):
        s = wl.quad_z(n, b)
        W, st = oracle.solve(s, scheme=scheme, tol=1e-7, max_steps=50000)
        assert st["converged"]
        Z, V = np.meshgrid(*s.coords(), indexing="ij")
        C = oracle.z_closed_form(Z, V, 0.91, 9.81, 19.62, 0.0, b, 0.5, 2.5)
        inner = (slice(4, -4), slice(4, -4))
        e = np.abs(W - C)[inner]
        hz = s.h()[0]
        assert e.max() < 2.0 * hz, (n, e.max())
        assert e.mean() < 0.05 * hz
        errs.append(e.mean())
        # sign of W away from the zero level set
        far = np.abs(C) > 2 * max(s.h())
        assert np.mean(np.sign(W[far]) == np.sign(C[far])) > 0.999
    assert errs[1] < 0.6 * errs[0]


@pytest.mark.parametrize("b", [0.5, 2.0])
def test_z_brute_force_game_brackets(b):
    """Fixed-horizon value at s = 0.3 against an exhaustive game tree with
    6 piecewise-constant intervals of bang-bang inputs, in both move orders."""
    zs = np.linspace(0.3, 2.7, 9)
    vs = np.linspace(-2.4, 2.4, 9)
    Z, V = np.meshgrid(zs, vs, indexing="ij")
    args = (Z, V, 0.3, 6, 0.91, 9.81, [0.0, 19.62], [-b, b], 0.5, 2.5)
    lo = oracle.brute_force_z(*args, disturbance_last=True)
    up = oracle.brute_force_z(*args, disturbance_last=False)
    assert np.all(lo <= up + 1e-12)
    s = wl.quad_z(201, b)
    k = int(math.ceil(0.3 / oracle.cfl_dt(s)))
    W, _ = oracle.solve(s, scheme=2, dt=0.3 / k, fixed_steps=k)
    iz = np.rint(Z / s.h()[0]).astype(int)
    iv = np.rint((V + 3.0) / s.h()[1]).astype(int)
    P = W[iz, iv]
    assert np.all(P >= lo - 0.02) and np.all(P <= up + 0.02)


@pytest.mark.parametrize("scheme", [2, 5])
def test_drift_1d_state_dependent_bound_closed_form(scheme):
    """Field |d| <= b0 + k|x| (Sec. II-C's state-dependent bound), safe |x| >= r:
    the disturbance drives the state toward 0 along y' = -(b0 + k y), so
    W(x, s) = max(y(s), 0) - r with y(s) = (|x| + b0/k) e^{-ks} - b0/k."""
    b0, k, r, T = 0.2, 0.5, 0.3, 0.5
    s = wl.drift((201,), 2.0, b0, wl.CON_BALL_OUT, r=r)
    x = s.coords()[0]
    b = b0 + k * np.abs(x)
    field = (-b[None, :], b[None, :])
    W, _ = oracle.solve(s, scheme=scheme, dt=T / 100, fixed_steps=100, dfield=field)
    y = (np.abs(x) + b0 / k) * np.exp(-k * T) - b0 / k
    exact = np.maximum(y, 0.0) - r
    h = s.h()[0]
    inner = slice(6, -6)
    assert np.abs(W - exact)[inner].max() < 2.0 * h
    away = np.abs(y) > 6 * h
    assert np.abs(W - exact)[away & (np.abs(x) < 1.9)].max() < 0.05 * h


@pytest.mark.parametrize("scheme", [2, 5])
def test_constraint_field_two_intervals_is_the_window_minimum(scheme):
    """Constraint given as an array (Sec. II-A, c for an arbitrary set C):
    a non-convex safe set, the union |x - 1| <= 0.5 or |x + 1.1| <= 0.6.
    With dx/dt = d, |d| <= b and no control, every point of
    [x - b s, x + b s] is reachable, so W(x, s) is the minimum of l over that
    window (found here by dense sampling)."""
    b, T = 0.4, 0.5
    s = wl.drift((241,), 2.5, b, wl.CON_BOX, r=1.0)
    x = s.coords()[0]

    def l_of(y):
        return np.maximum(0.5 - np.abs(y - 1.0), 0.6 - np.abs(y + 1.1))

    W, _ = oracle.solve(s, scheme=scheme, dt=T / 100, fixed_steps=100, lfield=l_of(x))
    ys = np.linspace(-b * T, b * T, 4001)
    exact = np.array([l_of(xi + ys).min() for xi in x])
    h = s.h()[0]
    inner = np.abs(x) < 2.5 - 6 * h
    assert np.abs(W - exact)[inner].max() < 2.0 * h
    # away from the kinks of the exact value the scheme is much closer: l
    # peaks at 1 and -1.1 and bottoms out at 0 in the gap, so the window
    # minimum has kinks at 1, -1.1 and +-b T
    kinks = np.array([1.0, -1.1, b * T, -b * T])
    far = inner & (np.abs(x[:, None] - kinks[None, :]).min(axis=1) > 12 * h)
    assert np.abs(W - exact)[far].max() < 1e-3 * h
    # the two pieces stay apart: the gap between them is unsafe
    assert W[np.argmin(np.abs(x + 0.2))] < 0


def test_constraint_field_equals_the_analytic_ball():
    """The same margin given as an array gives the same W as the analytic
    ball, and the closed form of the 1-D erosion."""
    s = wl.drift((37,), 2.0, 0.5, wl.CON_BALL_OUT, r=0.3)
    x = s.coords()[0]
    l = np.abs(x) - 0.3
    Wa, _ = oracle.solve(s, scheme=5, fixed_steps=20)
    Wf, _ = oracle.solve(s, scheme=5, fixed_steps=20, lfield=l)
    assert np.array_equal(Wa, Wf)
    assert np.array_equal(oracle.margin(s, l), l)


def test_safety_control_brakes_toward_the_safe_set():
    """The optimal safety control (Sec. II-A) on the z subsystem: near the
    ceiling while climbing it cuts thrust to its lower bound; near the floor
    while falling it applies full thrust (the braking curves of the double
    integrator).  The x subsystem near its +p face moving outward commands
    the lower input bound (tilt back), and the mirrored state the upper."""
    z = wl.quad_z(61, 0.5)
    Wz, st = oracle.solve(z, scheme=2, tol=1e-6, max_steps=50000)
    assert st["converged"]
    S = np.array([[2.3, 1.0], [0.7, -1.0]])
    u, w, act = oracle.safety_filter([z], [Wz], [(0, 1)], [0], S, np.full((2, 1), 9.0),
                                     level=10.0)
    assert u[:, 0].tolist() == [wl.Z_PARAMS[2], wl.Z_PARAMS[3]]
    assert act.tolist() == [1, 1]
    x = wl.quad_x4(11, 0.5)
    Wx, _ = oracle.solve(x, scheme=5, fixed_steps=200)
    X = np.array([[3.6, 1.5, 0.0, 0.0], [-3.6, -1.5, 0.0, 0.0]])
    u, w, act = oracle.safety_filter([x], [Wx], [(0, 1, 2, 3)], [0], X, np.zeros((2, 1)),
                                     level=0.5)
    assert u[:, 0].tolist() == [wl.X4_PARAMS[4], wl.X4_PARAMS[5]]


@pytest.mark.parametrize("make", [lambda: wl.quad_z(11, 0.5), lambda: wl.quad_x4(5, 0.5)])
def test_control_gain_matches_the_model(make):
    """The filter's df/du (per axis) agrees with the model that H is built
    on: raising the input's upper bound by du changes H(x, e_k) only on the
    controlled axis k, and there by gain_k du."""
    import dataclasses
    spec = make()
    b, ulo, uhi = oracle.control_gain(spec)
    iu = 3 if spec.model == wl.QUAD_Z else 5   # index of u_hi in the model parameters
    du = 0.25
    params = list(spec.params)
    params[iu] += du
    raised = dataclasses.replace(spec, params=tuple(params))
    x = [0.3, 0.2, 0.1, 0.05][:spec.ndim]
    for k in range(spec.ndim):
        e = [0.0] * spec.ndim
        e[k] = 1.0
        dH = oracle.hamiltonian(raised, x, e) - oracle.hamiltonian(spec, x, e)
        assert dH == pytest.approx(b[k] * du, abs=1e-12)
    assert b.any() and uhi == spec.params[iu]


def test_safety_filter_tie_keeps_the_clipped_performance_control():
    """Where the gradient along the input's axis is exactly zero (a value
    field constant along v), the performance control stays, clipped to the
    input box."""
    z = wl.quad_z(21, 0.5)
    zz = z.coords()[0]
    W = np.repeat((zz - 1.5)[:, None], 21, axis=1)  # W depends on z only
    S = np.array([[1.2, 0.4], [1.7, -0.3], [0.9, 0.0]])
    up = np.array([[25.0], [-3.0], [7.5]])
    u, w, act = oracle.safety_filter([z], [W], [(0, 1)], [0], S, up, level=10.0)
    assert act.tolist() == [1, 1, 1]
    assert u[:, 0].tolist() == [wl.Z_PARAMS[3], wl.Z_PARAMS[2], 7.5]


def test_safety_filter_switch_and_decomposed_value():
    """W = min over subsystems; the performance control passes where every
    W_k is above the level; each subsystem drives only its own input."""
    specs = [wl.demo10d_x(9, 0.5), wl.demo10d_x(9, 0.5, "y"), wl.demo10d_z(21, 0.5)]
    Ws = [oracle.solve(s, scheme=2, fixed_steps=30)[0] for s in specs]
    states = wl.quad10d_states(specs, 200, seed=3)
    up = np.tile([0.1, -0.1, 9.0], (200, 1))
    u, w, act = oracle.safety_filter(specs, Ws, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, states, up,
                                     level=-1e9)
    assert np.array_equal(u, up) and not act.any()
    vals = [oracle.query_value(s, W, states[:, list(a)])
            for s, W, a in zip(specs, Ws, wl.QUAD10D_AXES)]
    assert np.array_equal(w, np.minimum(np.minimum(vals[0], vals[1]), vals[2]))
    u, w, act = oracle.safety_filter(specs, Ws, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, states, up,
                                     level=0.0)
    for k in range(3):
        on = (act >> k) & 1 == 1
        assert np.array_equal(on, vals[k] <= 0.0)
        assert np.array_equal(u[~on, k], up[~on, k])


def test_translation_on_the_grid_is_an_index_shift():
    """A shift by whole cells moves the node values by whole indices; nodes
    whose source leaves the box take the cold start l."""
    z0 = wl.quad_z(61, 0.5, (0.5, 2.5))
    z1 = wl.quad_z(61, 0.5, (0.7, 2.7))
    W0 = oracle.margin(z0) + wl.seeded_field(z0, 5, 0.05)
    l1 = oracle.margin(z1)
    for k in (4, -3):
        shift = (k * z0.h()[0], 0.0)
        P = oracle.translate(z0, W0, z1, shift)
        moved = np.full_like(W0, np.inf)
        if k > 0:
            moved[k:] = W0[:-k]
        else:
            moved[:k] = W0[-k:]
        ref = np.minimum(np.where(np.isinf(moved), l1, moved), l1)
        assert np.abs(P - ref).max() < 1e-12


def test_translation_off_the_grid_is_linear_interpolation():
    """A move by a fraction of a cell reads the source by multilinear
    interpolation: the same as SciPy's linear grid interpolator at x - s,
    with the target's l where x - s leaves the source box, then min with l."""
    from scipy.interpolate import RegularGridInterpolator
    src = wl.quad_z(41, 0.5, (0.5, 2.5))
    dst = wl.quad_z(57, 0.5, (0.73, 2.73))
    Ws = oracle.margin(src) + wl.seeded_field(src, 9, 0.05)
    shift = (0.23, 0.0)
    P = oracle.translate(src, Ws, dst, shift)
    X = np.stack(np.meshgrid(*dst.coords(), indexing="ij"), axis=-1).reshape(-1, 2)
    Y = X - np.array(shift)
    inside = np.all((Y >= np.array(src.lo) - 1e-9) & (Y <= np.array(src.hi) + 1e-9), axis=1)
    f = RegularGridInterpolator(src.coords(), Ws, method="linear")
    ld = oracle.margin(dst).ravel()
    ref = ld.copy()
    ref[inside] = np.minimum(f(np.clip(Y[inside], src.lo, src.hi)), ld[inside])
    assert np.abs(P.ravel() - ref).max() < 1e-12
    assert (~inside).any() and inside.any()


def test_translated_prior_warm_start_is_exact():
    """The z dynamics do not depend on z, so the fixed point for a box moved
    along z is the moved fixed point: a warm start from the translated prior
    lands on the cold fixed point, in fewer steps (Sec. III-B)."""
    z0 = wl.quad_z(61, 0.5, (0.5, 2.5))
    z1 = wl.quad_z(61, 0.5, (0.7, 2.7))
    W0, _ = oracle.solve(z0, scheme=2, tol=1e-6, max_steps=50000)
    P = oracle.translate(z0, W0, z1, (0.2, 0.0))
    Wc, stc = oracle.solve(z1, scheme=2, tol=1e-6, max_steps=50000)
    Ww, stw = oracle.solve(z1, scheme=2, tol=1e-6, max_steps=50000, warm=P)
    assert stc["converged"] and stw["converged"]
    assert stw["steps"] < stc["steps"]
    assert np.abs(Ww - Wc).max() < 1e-5


def test_uniform_field_equals_box():
    s = wl.quad_x4(9, 0.6)
    W0, _ = oracle.solve(s, scheme=5, fixed_steps=4)
    f = (np.full((1,) + s.n, -0.6), np.full((1,) + s.n, 0.6))
    W1, _ = oracle.solve(s, scheme=5, fixed_steps=4, dfield=f)
    assert np.array_equal(W0, W1)
    assert np.array_equal(oracle.alpha(s), oracle.alpha(s, f))


def test_larger_field_gives_smaller_value():
    """Comparison principle: more disturbance anywhere can only lower W.
    First-order Lax-Friedrichs with one shared alpha is a monotone scheme, so
    this holds in the discrete iteration too.  Both fields peak at the same
    node (same alpha), and only nodes off the faces are checked: the linear
    ghost extrapolation 2 W_0 - W_1 is not monotone in W_1."""
    s = wl.quad_z(41, 0.3)
    small = wl.wind_field(s, 0.3, 1.5, 0, 0.6, 0.1)
    big = wl.wind_field(s, 0.3, 1.5, 0, 0.6, 0.4)
    assert np.array_equal(oracle.alpha(s, small), oracle.alpha(s, big))
    dt = 0.5 * oracle.cfl_dt(s, dfield=big)
    Ws, _ = oracle.solve(s, scheme=1, dt=dt, fixed_steps=80, dfield=small)
    Wb, _ = oracle.solve(s, scheme=1, dt=dt, fixed_steps=80, dfield=big)
    inner = (slice(1, -1), slice(1, -1))
    assert np.all(Wb[inner] <= Ws[inner] + 1e-12)
    assert (Ws - Wb)[inner].max() > 1e-2


# --------------------------------------------------------------- invariants

def test_tube_monotone_and_below_margin():
    s = wl.quad_z(61, 0.5)
    l = oracle.margin(s)
    prev = l.copy()
    for k in (5, 10, 20):
        W, _ = oracle.solve(s, scheme=2, fixed_steps=k, clamp=1)
        assert np.all(W <= l)
        assert np.all(W <= prev)
        prev = W
    Wvi, _ = oracle.solve(s, scheme=5, fixed_steps=20, clamp=0)
    assert np.all(Wvi <= l)


def test_fixed_point_independent_of_cfl():
    s = wl.quad_z(81, 0.5)
    W1, st1 = oracle.solve(s, scheme=2, cfl=0.5, tol=1e-8, max_steps=50000)
    W2, st2 = oracle.solve(s, scheme=2, cfl=0.25, tol=1e-8, max_steps=50000)
    assert st1["converged"] and st2["converged"]
    assert np.abs(W1 - W2).max() < 2e-3
    assert st2["steps"] > 1.8 * st1["steps"]


def test_warm_start_from_smaller_bound_reaches_cold_fixed_point():
    """Sec. III-B: a prior solved under a smaller disturbance set dominates the
    new fixed point, so the warm solve is sandwiched and lands on it."""
    s05 = wl.quad_z(101, 0.5)
    s10 = wl.quad_z(101, 1.0)
    Wp, _ = oracle.solve(s05, scheme=2, tol=1e-8, max_steps=50000)
    Wc, stc = oracle.solve(s10, scheme=2, tol=1e-8, max_steps=50000)
    Ww, stw = oracle.solve(s10, scheme=2, tol=1e-8, warm=Wp, max_steps=50000)
    assert stw["converged"]
    assert np.abs(Ww - Wc).max() < 1e-4 * np.abs(Wc).max()
    assert stw["steps"] < stc["steps"]


def test_warm_start_below_fixed_point_is_conservative():
    """A prior below the fixed point stays at or below it at every step (the
    iteration is monotone).  It creeps up only slowly, so the check stops
    early at 1e-5 per window."""
    s = wl.quad_z(61, 0.5)
    Wc, _ = oracle.solve(s, scheme=2, tol=1e-8, max_steps=50000)
    low = Wc - 0.2
    Ww, st = oracle.solve(s, scheme=2, tol=1e-5, warm=low, max_steps=50000)
    assert st["converged"]
    assert np.all(Ww <= Wc + 1e-6)


def test_x4_point_symmetry():
    """The 4-D subsystem is odd under (x, v, th, w) -> -(x, v, th, w) with a
    symmetric constraint and symmetric input boxes, so W is even under it."""
    s = wl.quad_x4(15, 0.5)
    W, _ = oracle.solve(s, scheme=5, fixed_steps=6)
    assert np.abs(W - W[::-1, ::-1, ::-1, ::-1]).max() < 1e-12
    assert np.abs(W - oracle.margin(s)).max() > 1e-3


def test_x_and_y_same_model_same_result():
    sx = wl.quad_x4(11, 0.5, 3.5, "x")
    sy = wl.quad_x4(11, 0.5, 3.5, "y")
    Wx, _ = oracle.solve(sx, scheme=5, fixed_steps=4)
    Wy, _ = oracle.solve(sy, scheme=5, fixed_steps=4)
    assert np.array_equal(Wx, Wy)


def test_band_stop_test_reduces_to_full_test_and_never_stops_later():
    """A band wider than max|W| is the full-grid test; a narrow band stops at
    the same window or earlier, with the zero level set already in place."""
    s = wl.quad_z(61, 0.5)
    Wf, stf = oracle.solve(s, scheme=2, tol=1e-4, max_steps=50000)
    Wb, stb = oracle.solve(s, scheme=2, tol=1e-4, band=100.0, max_steps=50000)
    assert stb["steps"] == stf["steps"] and np.array_equal(Wf, Wb)
    Wn, stn = oracle.solve(s, scheme=2, tol=1e-4, band=0.25, max_steps=50000)
    assert stn["converged"] and stn["steps"] <= stf["steps"]
    Wc, _ = oracle.solve(s, scheme=2, tol=1e-8, max_steps=50000)
    near = np.abs(Wc) < 0.25
    assert np.abs(Wn - Wc)[near].max() < 5e-3


def test_band_stop_test_stops_where_only_the_faces_still_move():
    """On a truncated 4-D grid the iterate keeps moving at the faces where
    trajectories leave the grid; the band test, which watches only
    |W| <= band around the zero level set, stops long before the full-grid
    test does."""
    s = wl.quad_x4(11, 0.8, 4.0, shift=0.5)
    Wb, stb = oracle.solve(s, scheme=5, tol=1e-4, clamp=1, band=0.5, max_steps=4000)
    assert stb["converged"] and stb["steps"] < 2500
    Wf, stf = oracle.solve(s, scheme=5, tol=1e-4, clamp=1, band=0.0, max_steps=4000)
    assert not stf["converged"] and stf["steps"] == 4000


def test_band_margin_skips_faces_of_free_axes_only():
    """The margin removes nodes next to faces of unconstrained axes from the
    stop test: on the 2-D z grid only the vz axis is free, so a margin wider
    than half that axis empties the test (it stops after one window), while
    a zero margin is the plain band test."""
    s = wl.quad_z(41, 0.5)
    W0, st0 = oracle.solve(s, scheme=2, tol=1e-4, band=0.5, max_steps=50000)
    W1, st1 = oracle.solve(s, scheme=2, tol=1e-4, band=0.5, band_margin=0, max_steps=50000)
    assert st0["steps"] == st1["steps"]
    W2, st2 = oracle.solve(s, scheme=2, tol=1e-4, band=0.5, band_margin=21, max_steps=50000)
    assert st2["windows"] == 1 and st2["residual"] == 0.0
    W3, st3 = oracle.solve(s, scheme=2, tol=1e-4, band=0.5, band_margin=3, max_steps=50000)
    assert st3["converged"] and st3["steps"] <= st0["steps"]


def test_no_motion_is_already_converged():
    s = wl.drift((11,), 1.0, 0.0, wl.CON_BOX, r=0.5)
    W, st = oracle.solve(s, scheme=2)
    assert st["converged"] and st["steps"] == 0
    assert np.array_equal(W, oracle.margin(s))


# ------------------------------------------------------ prolongation, query

def test_prolongation_exact_on_affine():
    big = dict(con_kind=wl.CON_BOX)
    c = wl.drift((7, 9), 2.0, 0.1, **big, r=100.0)
    f = wl.drift((13, 25), 2.0, 0.1, **big, r=100.0)
    X = np.meshgrid(*c.coords(), indexing="ij")
    Wc = 0.3 * X[0] - 0.7 * X[1] - 2.0
    Wf = oracle.prolong(c, Wc, f)
    Y = np.meshgrid(*f.coords(), indexing="ij")
    assert np.abs(Wf - (0.3 * Y[0] - 0.7 * Y[1] - 2.0)).max() < 1e-12


def test_prolongation_takes_min_with_margin():
    c = wl.quad_z(11, 0.5)
    f = wl.quad_z(21, 0.5)
    Wc = np.full(c.n, 10.0)
    Wf = oracle.prolong(c, Wc, f)
    assert np.array_equal(Wf, oracle.margin(f))


def test_prolongation_nonnested_4d_affine():
    """31^4 -> 81^4 is not nested (ratio 8/3); multilinear is still exact on affine fields."""
    c = wl.drift((5, 5, 5, 5), 1.0, 0.1, wl.CON_BOX, r=100.0)
    f = wl.drift((7, 7, 7, 7), 1.0, 0.1, wl.CON_BOX, r=100.0)
    X = np.meshgrid(*c.coords(), indexing="ij")
    a = [0.1, -0.2, 0.3, 0.4]
    Wc = sum(ai * xi for ai, xi in zip(a, X)) - 5.0
    Y = np.meshgrid(*f.coords(), indexing="ij")
    Wf = oracle.prolong(c, Wc, f)
    assert np.abs(Wf - (sum(ai * yi for ai, yi in zip(a, Y)) - 5.0)).max() < 1e-12


def test_query_value_and_gradient():
    s = wl.drift((11, 21), 1.0, 0.1, wl.CON_BOX, r=100.0)
    X = np.meshgrid(*s.coords(), indexing="ij")
    W = 2.0 * X[0] - 3.0 * X[1] + 0.5
    rng = np.random.default_rng(3)
    q = rng.uniform(-1.0, 1.0, size=(50, 2))
    v = oracle.query_value(s, W, q)
    assert np.allclose(v, 2.0 * q[:, 0] - 3.0 * q[:, 1] + 0.5, atol=1e-12)
    g = oracle.query_gradient(s, W, q)
    assert np.allclose(g, [[2.0, -3.0]] * 50, atol=1e-12)
    # quadratic: central differences are exact at interior nodes
    Wq = X[0] ** 2 + X[0] * X[1]
    nodes = np.array([[X[0][5, 7], X[1][5, 7]], [X[0][3, 12], X[1][3, 12]]])
    gq = oracle.query_gradient(s, Wq, nodes)
    assert np.allclose(gq, [[2 * n[0] + n[1], n[0]] for n in nodes], atol=1e-12)
    with pytest.raises(ValueError):
        oracle.query_value(s, W, np.array([[1.5, 0.0]]))
