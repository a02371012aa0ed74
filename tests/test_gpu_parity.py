"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerance: |W_gpu - W_oracle| <= 1e-4 * max|W_oracle|.  The sign of W must
agree at >= 99.99 % of the nodes that lie more than one cell from the oracle's
zero level set.  Both bounds come from the accuracy target for this solve.
Fixed-horizon cases give both sides the same dt and the same step count.
Converged 2-D cases run the oracle to a 1e-7 window residual and the GPU to
1e-5, its FP32 floor; converged 4-D cases use the 1e-4 stop rule on both sides.
"""

import numpy as np
import pytest

import oracle
from paper_2101_05916_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REL = 1e-4
SIGN_FRAC = 0.9999


@pytest.fixture(scope="module")
def hj():
    import torch
    assert torch.cuda.is_available()
    from paper_2101_05916_gb300 import build, hj as hjmod
    build.build()
    hjmod.lib()
    return hjmod


def assert_parity(Wg, Wo, spec, rel=REL):
    Wg = np.asarray(Wg, dtype=np.float64).reshape(Wo.shape)
    scale = np.abs(Wo).max()
    err = np.abs(Wg - Wo).max()
    assert err <= rel * scale, "max err %.3e > %.1e * %.3e" % (err, rel, scale)
    # sign test away from the zero level set (more than one cell in every axis)
    near = np.zeros(Wo.shape, dtype=bool)
    pos = Wo >= 0
    for ax in range(Wo.ndim):
        for sh in (1, -1):
            rolled = np.roll(pos, sh, axis=ax)
            edge = [slice(None)] * Wo.ndim
            edge[ax] = slice(0, 1) if sh == 1 else slice(-1, None)
            diff = rolled != pos
            diff[tuple(edge)] = False
            near |= diff
    far = ~near & (Wo != 0)
    if far.any():
        agree = np.mean(np.sign(Wg[far]) == np.sign(Wo[far]))
        assert agree >= SIGN_FRAC, "sign agreement %.6f" % agree


def gpu_fixed(hj, spec, scheme, steps, dt=None, clamp=0, warm=None):
    g = hj.Grid.from_spec(spec)
    try:
        if warm is not None:
            g.set_value(np.ascontiguousarray(warm, dtype=np.float32))
        if dt is None:
            dt = oracle.cfl_dt(spec)
        st = g.solve(hj.HJ_WARM if warm is not None else hj.HJ_COLD, scheme=scheme, dt=dt,
                     fixed_steps=steps, clamp=clamp)
        return g.value(), st
    finally:
        g.close()


CASES_FIXED = [
    ("z101_eno2", lambda: wl.quad_z(101, 0.5), 2, 60),
    ("z101_weno5", lambda: wl.quad_z(101, 0.5), 5, 60),
    ("z101_first", lambda: wl.quad_z(101, 0.5), 1, 60),
    ("z57x83_asym", lambda: wl.dataclasses.replace(wl.quad_z(57, 0.0), n=(57, 83),
                                                   d_lo=(-1.2,), d_hi=(0.3,)), 5, 40),
    ("x21_weno5", lambda: wl.quad_x4(21, 0.5), 5, 12),
    ("x21_eno2", lambda: wl.quad_x4(21, 0.5), 2, 12),
    ("x17_axis1", lambda: wl.dataclasses.replace(
        wl.quad_x4(17, 0.7), params=wl.X4_PARAMS[:6] + (1.0,)), 5, 10),
    ("x13x15x9x19_ragged", lambda: wl.quad_x4(13, 0.5).with_grid((13, 15, 9, 19)), 5, 10),
    ("drift1_ball", lambda: wl.drift((37,), 2.0, 0.5, wl.CON_BALL_OUT, r=0.3), 5, 20),
    ("drift2_box", lambda: wl.drift((23, 29), 2.0, 0.4, wl.CON_BOX, r=1.1), 5, 20),
    ("drift3_ball", lambda: wl.drift((11, 13, 17), 2.0, 0.4, wl.CON_BALL_OUT, r=0.5), 2, 15),
    ("drift4_box", lambda: wl.drift((7, 9, 11, 13), 2.0, 0.3, wl.CON_BOX, r=1.0), 5, 10),
    ("drift4_min3", lambda: wl.drift((3, 3, 3, 3), 1.0, 0.3, wl.CON_BOX, r=0.5), 5, 5),
]


@pytest.mark.parametrize("name,make,scheme,steps", CASES_FIXED, ids=[c[0] for c in CASES_FIXED])
def test_fixed_horizon_parity(hj, name, make, scheme, steps):
    spec = make()
    dt = oracle.cfl_dt(spec)
    Wo, _ = oracle.solve(spec, scheme=scheme, dt=dt, fixed_steps=steps)
    Wg, st = gpu_fixed(hj, spec, scheme, steps, dt=dt)
    assert st["steps"] == steps
    assert_parity(Wg, Wo, spec)


@pytest.mark.parametrize("name,make,scheme,steps,axis,centre", [
    ("z101_fan", lambda: wl.quad_z(101, 0.3), 2, 50, 0, 0.5),
    ("x21_wall", lambda: wl.quad_x4(21, 0.3), 5, 10, 0, 3.0),
])
def test_state_dependent_bound_parity(hj, name, make, scheme, steps, axis, centre):
    """GP-like state-dependent wind (Sec. II-C): base 0.3 plus a Gaussian bump."""
    spec = make()
    field = wl.wind_field(spec, 0.3, 1.5, axis, centre, 0.5)
    dt = oracle.cfl_dt(spec, dfield=field)
    Wo, _ = oracle.solve(spec, scheme=scheme, dt=dt, fixed_steps=steps, dfield=field)
    g = hj.Grid.from_spec(spec)
    g.set_disturbance_field(field[0], field[1])
    assert np.allclose(g.alpha(), oracle.alpha(spec, field), rtol=2e-7, atol=1e-7)
    st = g.solve(hj.HJ_COLD, scheme=scheme, dt=dt, fixed_steps=steps)
    Wg = g.value()
    # a box bound afterwards replaces the field again
    g.set_disturbance_bound([-0.3], [0.3])
    assert np.allclose(g.alpha(), oracle.alpha(spec.with_bound(0.3)), rtol=2e-7)
    g.close()
    assert_parity(Wg, Wo, spec)


@pytest.mark.parametrize("name,make,scheme,steps", [
    ("demo10d_x17", lambda: wl.demo10d_x(17, 0.5), 5, 10),
    ("demo10d_z101", lambda: wl.demo10d_z(101, 0.5), 2, 60),
])
def test_multi_axis_box_parity(hj, name, make, scheme, steps):
    """The 10-D demo's constraint boxes span several axes of a subsystem."""
    spec = make()
    dt = oracle.cfl_dt(spec)
    Wo, _ = oracle.solve(spec, scheme=scheme, dt=dt, fixed_steps=steps)
    Wg, st = gpu_fixed(hj, spec, scheme, steps, dt=dt)
    assert_parity(Wg, Wo, spec)


def test_constraint_field_parity(hj):
    """Non-convex safe set given as an array: z in [0.5, 1.4] or [1.6, 2.5]."""
    spec = wl.quad_z(101, 0.5)
    l = wl.two_band_margin(spec, [(0.5, 1.4), (1.6, 2.5)])
    dt = oracle.cfl_dt(spec)
    g = hj.Grid.from_spec(spec)
    g.set_constraint_field(l)
    for scheme, steps in ((5, 60), (2, 60)):
        Wo, _ = oracle.solve(spec, scheme=scheme, dt=dt, fixed_steps=steps, lfield=l)
        g.solve(hj.HJ_COLD, scheme=scheme, dt=dt, fixed_steps=steps)
        assert_parity(g.value(), Wo, spec)
    # converged at 1e-4 per window, ENO2 with the VI clamp (stencil switching
    # at the inner faces holds the residual near 1e-5, so no tighter stop);
    # W is compared with the oracle at the GPU's own stop step
    Wo, sto = oracle.solve(spec, scheme=2, dt=dt, tol=1e-4, max_steps=50000, lfield=l)
    st = g.solve(hj.HJ_COLD, scheme=2, dt=dt, tol=1e-4)
    assert st["converged"] and sto["converged"]
    assert abs(st["windows"] - sto["windows"]) <= 6
    Wc = g.value()
    Wt, _ = oracle.solve(spec, scheme=2, dt=dt, fixed_steps=st["steps"], lfield=l)
    assert_parity(Wc, Wt, spec)
    # the gap between the bands is never safe, and W <= l everywhere
    assert np.all(Wc <= l.astype(np.float32) + 1e-6)
    z = spec.coords()[0]
    assert np.all(Wc[(z > 1.4) & (z < 1.6)] < 0)
    # a box afterwards replaces the array
    g.solve(hj.HJ_COLD, scheme=2, dt=dt, fixed_steps=5)
    hj.hj_set_constraint(g.handle, spec.con_a, spec.con_b)
    g.solve(hj.HJ_COLD, scheme=2, dt=dt, fixed_steps=5)
    Wb = g.value()
    Wo, _ = oracle.solve(spec, scheme=2, dt=dt, fixed_steps=5)
    assert_parity(Wb, Wo, spec)
    g.close()


def test_constraint_field_prolong_and_errors(hj):
    cs, fs = wl.quad_z(51, 0.5), wl.quad_z(101, 0.5)
    lc = wl.two_band_margin(cs, [(0.5, 1.4), (1.6, 2.5)])
    lf = wl.two_band_margin(fs, [(0.5, 1.4), (1.6, 2.5)])
    gc, gf = hj.Grid.from_spec(cs), hj.Grid.from_spec(fs)
    gc.set_constraint_field(lc)
    gf.set_constraint_field(lf)
    gc.solve(hj.HJ_COLD, scheme=2, fixed_steps=40)
    Wc = gc.value()
    hj.prolong(gc, gf)
    Wo = oracle.prolong(cs, Wc.astype(np.float64), fs, lfield_fine=lf)
    assert np.abs(gf.value() - Wo).max() <= 1e-5 * np.abs(Wo).max()
    with pytest.raises(ValueError):
        gf.set_constraint_field(lf[:10])
    bad = lf.copy()
    bad[3, 4] = np.inf
    with pytest.raises(hj.HJError):
        gf.set_constraint_field(bad)
    with pytest.raises(hj.HJError) as e:
        gf.solve(hj.HJ_COLD, scheme=2, fixed_steps=2)
    assert e.value.status == hj.HJ_ERR_STATE
    gc.close()
    gf.close()


def test_safety_filter_parity(hj):
    """Decomposed 10-D safety filter (Sec. II-A, II-B, III-A) on the GPU
    against the oracle's filter, on the same float32 value grids."""
    specs = [wl.demo10d_x(15, 0.5), wl.demo10d_x(13, 0.7, "y"), wl.demo10d_z(61, 0.5)]
    Ws = [oracle.solve(s, scheme=5 if s.ndim == 4 else 2, fixed_steps=40)[0].astype(np.float32)
          for s in specs]
    grids = []
    for s, W in zip(specs, Ws):
        g = hj.Grid.from_spec(s)
        g.set_value(W)
        grids.append(g)
    states = wl.quad10d_states(specs, 20000, seed=11)
    up = np.tile([0.05, -0.05, 9.0], (states.shape[0], 1))
    W64 = [W.astype(np.float64) for W in Ws]
    for level in (0.0, 0.3):
        u, w, act = hj.hj_safety_filter(grids, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, states, up, level)
        uo, wo, ao = oracle.safety_filter(specs, W64, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, states,
                                          up, level)
        assert np.abs(w - wo).max() <= 1e-9 * np.abs(wo).max()
        # switching and bang-bang decisions are unique away from exact ties
        vals = [oracle.query_value(s, W, states[:, list(a)])
                for s, W, a in zip(specs, W64, wl.QUAD10D_AXES)]
        grads = [oracle.query_gradient(s, W, states[:, list(a)])
                 for s, W, a in zip(specs, W64, wl.QUAD10D_AXES)]
        for k, s in enumerate(specs):
            b, _, _ = oracle.control_gain(s)
            gain = grads[k] @ b
            clear = (np.abs(vals[k] - level) > 1e-9) & (np.abs(gain) > 1e-9)
            assert np.array_equal(((act >> k) & 1)[clear], ((ao >> k) & 1)[clear])
            assert np.array_equal(u[clear, k], uo[clear, k])
        assert act.any() and (act == 0).any()
    # device buffers on the grids' stream
    import torch
    ts, tu = torch.from_numpy(states).cuda(), torch.from_numpy(up).cuda()
    ud, wd, ad = hj.hj_safety_filter(grids, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, ts, tu, 0.0)
    u0, w0, a0 = hj.hj_safety_filter(grids, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, states, up, 0.0)
    assert np.array_equal(ud.cpu().numpy(), u0) and np.array_equal(wd.cpu().numpy(), w0)
    assert np.array_equal(ad.cpu().numpy(), a0)
    # the prepared filter object gives the same result, state by state
    filt = hj.SafetyFilter(grids, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, 10, 3, max_states=4)
    uf, wf, af = filt(np.ascontiguousarray(states[:4]), np.ascontiguousarray(up[:4]), 0.0)
    assert np.array_equal(uf, u0[:4]) and np.array_equal(wf, w0[:4]) and np.array_equal(af, a0[:4])
    # errors: a state outside a box, a control driven twice
    bad = states[:4].copy()
    bad[0, 0] = 100.0
    with pytest.raises(hj.HJError):
        hj.hj_safety_filter(grids, wl.QUAD10D_AXES, wl.QUAD10D_CTRL, bad, up[:4], 0.0)
    with pytest.raises(hj.HJError):
        hj.hj_safety_filter(grids, wl.QUAD10D_AXES, (0, 0, 2), states[:4], up[:4], 0.0)
    for g in grids:
        g.close()


def test_translate_parity_and_errors(hj):
    """hj_translate against the oracle: non-aligned shifts along the position
    axis, resolution change, and nodes whose source leaves the box."""
    cases = [(wl.quad_z(41, 0.5, (0.5, 2.5)), wl.quad_z(67, 0.7, (0.83, 2.83)), (0.33, 0.0)),
             (wl.quad_x4(13, 0.5), wl.quad_x4(15, 0.5, shift=-0.7), (-0.7, 0.0, 0.0, 0.0))]
    for src, dst, shift in cases:
        Ws = (oracle.margin(src) + wl.seeded_field(src, 3, 0.05)).astype(np.float32)
        gs, gd = hj.Grid.from_spec(src), hj.Grid.from_spec(dst)
        gs.set_value(Ws)
        hj.translate(gs, gd, shift)
        Wo = oracle.translate(src, Ws.astype(np.float64), dst, shift)
        assert np.abs(gd.value() - Wo).max() <= 1e-6 * np.abs(Wo).max()
        bad_shift = list(shift)
        bad_shift[1] = 0.1
        with pytest.raises(hj.HJError):
            hj.translate(gs, gd, bad_shift)
        with pytest.raises(hj.HJError):
            hj.translate(gs, gs, shift)
        gs.close()
        gd.close()
    # a state-dependent disturbance bound breaks translation invariance
    z = wl.quad_z(21, 0.5)
    g1, g2 = hj.Grid.from_spec(z), hj.Grid.from_spec(z)
    g1.solve(hj.HJ_COLD, scheme=2, fixed_steps=2)
    g2.set_disturbance_field(*wl.wind_field(z, 0.5, 0.2, 0, 1.0, 0.5))
    with pytest.raises(hj.HJError) as e:
        hj.translate(g1, g2, (0.1, 0.0))
    assert e.value.status == hj.HJ_ERR_STATE
    g1.close()
    g2.close()


def test_translated_warm_start_reaches_cold_fixed_point(hj):
    z0 = wl.quad_z(101, 0.5, (0.5, 2.5))
    z1 = wl.quad_z(101, 0.5, (0.65, 2.65))
    g0, g1 = hj.Grid.from_spec(z0), hj.Grid.from_spec(z1)
    g0.solve(hj.HJ_COLD, scheme=2, tol=1e-5)
    hj.translate(g0, g1, (0.15, 0.0))
    warm = g1.solve(hj.HJ_WARM, scheme=2, tol=1e-5)
    Ww = g1.value()
    cold = g1.solve(hj.HJ_COLD, scheme=2, tol=1e-5)
    Wc = g1.value()
    g0.close()
    g1.close()
    assert warm["converged"] and cold["converged"] and warm["steps"] < cold["steps"]
    assert np.abs(Ww - Wc).max() <= 1e-4 * np.abs(Wc).max()


def test_monotone_clamp_parity(hj):
    spec = wl.quad_z(61, 0.8)
    dt = oracle.cfl_dt(spec)
    Wo, _ = oracle.solve(spec, scheme=5, dt=dt, fixed_steps=40, clamp=1)
    Wg, _ = gpu_fixed(hj, spec, 5, 40, dt=dt, clamp=1)
    assert_parity(Wg, Wo, spec)
    l = oracle.margin(spec)
    assert np.all(Wg <= l.astype(np.float32) + 1e-6)


def test_warm_start_from_seeded_prior_parity(hj):
    spec = wl.quad_x4(15, 0.5)
    prior = oracle.margin(spec) + 0.3 * wl.seeded_field(spec, 11, 0.2)
    dt = oracle.cfl_dt(spec)
    Wo, _ = oracle.solve(spec, scheme=5, dt=dt, fixed_steps=8, warm=prior)
    Wg, _ = gpu_fixed(hj, spec, 5, 8, dt=dt, warm=prior)
    assert_parity(Wg, Wo, spec)


def test_alpha_parity(hj):
    for spec in (wl.config0(), wl.config1(), wl.drift((5, 7), 1.0, 0.3),
                 wl.dataclasses.replace(wl.quad_z(11, 0.0), d_lo=(-0.2,), d_hi=(1.7,))):
        g = hj.Grid.from_spec(spec)
        a = g.alpha()
        g.close()
        assert np.allclose(a, oracle.alpha(spec), rtol=2e-7, atol=1e-7)


def test_z101_converged_parity(hj):
    spec = wl.config0()
    Wo, sto = oracle.solve(spec, scheme=2, tol=1e-7, max_steps=50000)
    g = hj.Grid.from_spec(spec)
    st = g.solve(hj.HJ_COLD, scheme=2, tol=1e-5)
    Wg = g.value()
    g.close()
    assert st["converged"] and sto["converged"]
    assert_parity(Wg, Wo, spec)


def test_z101_converged_default_tol_matches_oracle_window_count(hj):
    """At the configuration's own stop rule (1e-4 per 0.1 s) both sides stop
    after the same number of windows."""
    spec = wl.config0()
    Wo, sto = oracle.solve(spec, scheme=2, tol=1e-4, max_steps=50000)
    g = hj.Grid.from_spec(spec)
    st = g.solve(hj.HJ_COLD, scheme=2, tol=1e-4)
    Wg = g.value()
    g.close()
    assert st["converged"]
    assert abs(st["windows"] - sto["windows"]) <= 1
    assert np.abs(Wg - Wo).max() <= 1e-3 * np.abs(Wo).max()


def converged_4d(hj, spec, **kw):
    """Both sides run the stop rule at the same dt.  Near tol = 1e-4 the window
    residual of these grids falls by only about 7e-7 per 0.1 s window, so the
    FP32 rounding of the two snapshots (a few 1e-6) can move the GPU's stop a
    few windows from the oracle's.  W is then compared with the oracle at the
    GPU's own stop step."""
    dt = oracle.cfl_dt(spec)
    Wo, sto = oracle.solve(spec, dt=dt, max_steps=60000, **kw)
    g = hj.Grid.from_spec(spec)
    st = g.solve(hj.HJ_COLD, dt=dt, **kw)
    Wg = g.value()
    g.close()
    assert st["converged"] and sto["converged"]
    assert abs(st["windows"] - sto["windows"]) <= 6, (st["windows"], sto["windows"])
    kw_fixed = {k: v for k, v in kw.items() if k not in ("tol", "band", "band_margin")}
    Wt, _ = oracle.solve(spec, dt=dt, fixed_steps=st["steps"], **kw_fixed)
    assert_parity(Wg, Wt, spec)


def test_x13_converged_parity(hj):
    """4-D, converged at the configuration's own stop rule (1e-4 per 0.1 s)."""
    converged_4d(hj, wl.quad_x4(13, 0.5), scheme=5, tol=1e-4)


def test_x13_converged_parity_monotone_band(hj):
    """The 4-D workload setting: monotone clamp, band stop test."""
    converged_4d(hj, wl.quad_x4(13, 0.8, 4.0, shift=0.5), scheme=5, tol=1e-4, clamp=1, band=0.5)


def test_x17_converged_parity_vi_band_margin(hj):
    """VI clamp with the band stop test skipping a 3-cell layer at the faces
    of the free axes (v, theta, omega), both sides."""
    converged_4d(hj, wl.quad_x4(17, 0.8, 4.0, shift=0.5), scheme=5, tol=1e-4, clamp=0, band=0.5,
                 band_margin=3)


def test_warm_start_reaches_cold_fixed_point(hj):
    """Sec. III-B on the GPU: the b = 0.5 result warm-starts the b = 1.0 solve,
    which lands on the cold b = 1.0 fixed point in fewer steps."""
    s05, s10 = wl.quad_z(101, 0.5), wl.quad_z(101, 1.0)
    g = hj.Grid.from_spec(s05)
    g.solve(hj.HJ_COLD, scheme=2, tol=1e-6)
    g.set_disturbance_bound([-1.0], [1.0])
    warm = g.solve(hj.HJ_WARM, scheme=2, tol=1e-6)
    Ww = g.value()
    cold = g.solve(hj.HJ_COLD, scheme=2, tol=1e-6)
    Wc = g.value()
    g.close()
    assert warm["converged"] and cold["converged"]
    assert warm["steps"] < cold["steps"]
    assert np.abs(Ww - Wc).max() <= REL * np.abs(Wc).max()
    Wo, _ = oracle.solve(s10, scheme=2, tol=1e-7, max_steps=50000)
    assert_parity(Ww, Wo, s10)


def test_local_wind_increase_warm_start(hj):
    """A local (GP-like) rise of the wind bound: the fixed point under the
    base field dominates the new one, so warm-starting from it reaches the
    cold fixed point under the raised field (Sec. III-B), and both match the
    oracle solved with the same field."""
    spec = wl.quad_z(101, 0.3)
    base = wl.wind_field(spec, 0.3, 0.0, 0, 1.5, 0.4)
    raised = wl.wind_field(spec, 0.3, 1.2, 0, 2.2, 0.3)
    g = hj.Grid.from_spec(spec)
    g.set_disturbance_field(*base)
    g.solve(hj.HJ_COLD, scheme=2, tol=1e-5, max_steps=50000)
    g.set_disturbance_field(*raised)
    warm = g.solve(hj.HJ_WARM, scheme=2, tol=1e-5, max_steps=50000)
    Ww = g.value()
    cold = g.solve(hj.HJ_COLD, scheme=2, tol=1e-5, max_steps=50000)
    Wc = g.value()
    g.close()
    assert warm["converged"] and cold["converged"]
    assert warm["steps"] < cold["steps"]
    assert np.abs(Ww - Wc).max() <= REL * np.abs(Wc).max()
    # ENO2 stencil switching near the bump holds the window residual near
    # 1e-6 here, so both sides stop at 1e-5 per 0.1 s
    Wo, sto = oracle.solve(spec, scheme=2, tol=1e-5, dfield=raised, max_steps=50000)
    assert sto["converged"]
    assert_parity(Ww, Wo, spec)


def test_field_errors(hj):
    spec = wl.quad_z(11, 0.3)
    g = hj.Grid.from_spec(spec)
    lo, hi = wl.wind_field(spec, 0.3, 0.5, 0, 1.0, 0.5)
    with pytest.raises(hj.HJError):
        g.set_disturbance_field(hi, lo)         # lo > hi somewhere
    with pytest.raises(ValueError):
        g.set_disturbance_field(lo[:, :5], hi[:, :5])
    bad = hi.copy()
    bad[0, 3, 4] = np.nan
    with pytest.raises(hj.HJError):
        g.set_disturbance_field(lo, bad)
    # after a rejected field no bound is in force until one is set
    with pytest.raises(hj.HJError) as e:
        g.solve(hj.HJ_COLD, scheme=2, fixed_steps=2)
    assert e.value.status == hj.HJ_ERR_STATE
    g.set_disturbance_bound([-0.3], [0.3])
    assert np.allclose(g.alpha(), oracle.alpha(spec), rtol=2e-7)
    g.close()


def test_prolongation_parity(hj):
    c, f = wl.quad_x4(11, 1.0), wl.quad_x4(27, 1.0)
    Wc = (oracle.margin(c) + wl.seeded_field(c, 5, 0.1)).astype(np.float32)
    gc, gf = hj.Grid.from_spec(c), hj.Grid.from_spec(f)
    gc.set_value(Wc)
    hj.prolong(gc, gf)
    Wf = gf.value()
    gc.close()
    gf.close()
    Wo = oracle.prolong(c, Wc.astype(np.float64), f)
    assert np.abs(Wf - Wo).max() <= 2e-6 * np.abs(Wo).max()


def test_prolongation_outside_coarse_box_is_rejected(hj):
    c = wl.quad_z(11, 0.5)
    f = wl.dataclasses.replace(wl.quad_z(11, 0.5), hi=(3.5, 3.0))
    gc, gf = hj.Grid.from_spec(c), hj.Grid.from_spec(f)
    gc.solve(hj.HJ_COLD, scheme=2, fixed_steps=1)
    with pytest.raises(hj.HJError) as e:
        hj.prolong(gc, gf)
    assert e.value.status == hj.HJ_ERR_ARG
    gc.close()
    gf.close()


def test_query_parity(hj):
    spec = wl.quad_x4(13, 0.5)
    W = (oracle.margin(spec) + wl.seeded_field(spec, 9, 0.05)).astype(np.float32)
    g = hj.Grid.from_spec(spec)
    g.set_value(W)
    rng = np.random.default_rng(4)
    xs = rng.uniform(spec.lo, spec.hi, size=(257, 4))
    v = g.query_value(xs)
    gr = g.query_gradient(xs)
    with pytest.raises(hj.HJError):
        g.query_value(np.array([[6.0, 0, 0, 0]]))
    assert g.query_value(np.zeros((0, 4))).shape == (0,)
    g.close()
    W64 = W.astype(np.float64)
    assert np.allclose(v, oracle.query_value(spec, W64, xs), rtol=1e-12, atol=1e-12)
    assert np.allclose(gr, oracle.query_gradient(spec, W64, xs), rtol=1e-10, atol=1e-10)


def test_batch_equals_single_grid_bitwise(hj):
    """The fused multi-grid launch runs the same per-node code, so every grid
    of a batch ends bit-identical to its own single-grid solve."""
    specs = [wl.quad_x4(17, 0.5, 4.0, "x"), wl.quad_x4(17, 0.5, 3.5, "y"), wl.quad_z(61, 0.5)]
    schemes = [5, 5, 2]
    singles = []
    for s, sc in zip(specs, schemes):
        g = hj.Grid.from_spec(s)
        st = g.solve(hj.HJ_COLD, scheme=sc, tol=1e-4, max_steps=3000)
        singles.append((g.value(), st))
        g.close()
    grids = [hj.Grid.from_spec(s) for s in specs]
    opts = [hj.make_opts(scheme=sc, tol=1e-4, max_steps=3000) for sc in schemes]
    rc, statuses, stats = hj.hj_solve_batch([g.handle for g in grids], [0, 0, 0], opts)
    for g, (Ws, sts), stb in zip(grids, singles, stats):
        Wb = g.value()
        assert stb["steps"] == sts["steps"]
        assert np.array_equal(Wb, Ws)
        g.close()


def test_group_launch_is_one_launch_per_stage_and_bitwise_equal(hj):
    """Once the group kernels of a batch's composition are compiled, every
    RK stage of every active grid, whatever its kind, is one launch (plus
    one control launch per step), and each grid still ends bit-identical to
    its own single-grid solve: fixed steps and to convergence."""
    specs = [wl.quad_x4(17, 0.5, 4.0, "x"), wl.quad_x4(17, 0.5, 3.5, "y"), wl.quad_z(61, 0.5),
             wl.quad_x4(13, 0.3)]
    schemes = [5, 5, 2, 5]
    grids = [hj.Grid.from_spec(s) for s in specs]
    opts = [hj.make_opts(scheme=sc, fixed_steps=2) for sc in schemes]
    hj.hj_solve_batch([g.handle for g in grids], [0] * 4, opts)  # starts the group compile
    assert hj.hj_jit_wait(120.0)
    for fixed in (37, 0):
        singles = []
        for s, sc in zip(specs, schemes):
            g = hj.Grid.from_spec(s)
            st = g.solve(hj.HJ_COLD, scheme=sc, fixed_steps=fixed, tol=1e-4, max_steps=3000)
            singles.append((g.value(), st))
            g.close()
        opts = [hj.make_opts(scheme=sc, fixed_steps=fixed, tol=1e-4, max_steps=3000)
                for sc in schemes]
        before = hj.hj_kernel_launches()
        rc, statuses, stats = hj.hj_solve_batch([g.handle for g in grids], [0] * 4, opts)
        launches = hj.hj_kernel_launches() - before
        # converged runs of the 4-D grids may reach the step cap (VI clamp,
        # full-grid test: the truncated faces keep moving); the single-grid
        # solves reach the same cap at the same step
        ok = (hj.HJ_OK,) if fixed else (hj.HJ_OK, hj.HJ_ERR_NOT_CONVERGED)
        assert all(st in ok for st in statuses), (rc, statuses, hj.hj_last_error())
        if fixed:
            # 4 inits, then 3 group launches and 1 control launch per step
            assert launches == 4 + 4 * fixed, launches
        for g, (Ws, sts), stb in zip(grids, singles, stats):
            assert stb["steps"] == sts["steps"]
            assert np.array_equal(g.value(), Ws)
    for g in grids:
        g.close()


def test_allocator_hook_serves_grid_memory_from_torch(hj):
    """hj_set_allocator routes a grid's device memory through PyTorch's
    caching allocator: the grid's fields show up in torch's allocated bytes
    while it lives and leave with it, and the solve is unchanged bit for
    bit."""
    import torch
    spec = wl.quad_x4(17, 0.5)
    g = hj.Grid.from_spec(spec)
    g.solve(hj.HJ_COLD, scheme=5, fixed_steps=9)
    ref = g.value()
    g.close()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    hj.use_torch_allocator(True)
    try:
        g = hj.Grid.from_spec(spec)
        during = torch.cuda.memory_allocated()
        g.solve(hj.HJ_COLD, scheme=5, fixed_steps=9)
        W = g.value()
        g.close()
        torch.cuda.synchronize()
        after = torch.cuda.memory_allocated()
    finally:
        hj.use_torch_allocator(False)
    assert during - before >= 4 * spec.npts * 4
    assert after == before
    assert np.array_equal(W, ref)


def test_x_and_y_identical_inputs_identical_results(hj):
    s = wl.quad_x4(15, 0.5, 3.5)
    a, b = hj.Grid.from_spec(s), hj.Grid.from_spec(s)
    rc, _, st = hj.hj_solve_batch([a.handle, b.handle], [0, 0], [hj.make_opts(fixed_steps=30)])
    assert np.array_equal(a.value(), b.value())
    a.close()
    b.close()


# ------------------------------------------------------------ full sizes

def test_config1_full_size_fixed_horizon(hj):
    """41^4, WENO5, five steps from the cold start, with the kernels the
    bench times: the stage kernels specialised to the 41^4 grid (their
    background compile is started and awaited first), and the precompiled
    ones."""
    spec = wl.config1()
    dt = oracle.cfl_dt(spec)
    Wo, _ = oracle.solve(spec, scheme=5, dt=dt, fixed_steps=5)
    gpu_fixed(hj, spec, 5, 1, dt=dt)
    assert hj.hj_jit_wait(120.0)
    before = hj.hj_jit_kernels()
    launches = hj.hj_kernel_launches()
    Wg, _ = gpu_fixed(hj, spec, 5, 5, dt=dt)
    assert hj.hj_kernel_launches() > launches
    assert hj.hj_jit_kernels() >= before and hj.hj_jit_kernels() > 0
    assert_parity(Wg, Wo, spec)
    try:
        hj.hj_set_jit(False)
        Wp, _ = gpu_fixed(hj, spec, 5, 5, dt=dt)
    finally:
        hj.hj_set_jit(True)
    assert np.array_equal(Wg, Wp)


def test_config2_batch_full_size_fixed_horizon(hj):
    """x, y at 61^4 and z at 201^2 as one fused batch, two steps each, sampled
    against the oracle on every node of each grid."""
    specs = [s.with_bound(0.5) for s in wl.config2()]
    schemes = [5, 5, 2]
    grids = [hj.Grid.from_spec(s) for s in specs]
    dts = [oracle.cfl_dt(s) for s in specs]
    opts = [hj.make_opts(scheme=sc, dt=dt, fixed_steps=2) for sc, dt in zip(schemes, dts)]
    rc, statuses, stats = hj.hj_solve_batch([g.handle for g in grids], [0, 0, 0], opts)
    assert all(s == 0 for s in statuses)
    for g, s, sc, dt in zip(grids, specs, schemes, dts):
        Wo, _ = oracle.solve(s, scheme=sc, dt=dt, fixed_steps=2)
        assert_parity(g.value(), Wo, s)
        g.close()


def test_config3_prolong_full_size_sampled(hj):
    """31^4 -> 81^4 prolongation of a seeded coarse field, checked against the
    oracle's interpolation at 4096 sampled fine nodes."""
    c, f, _ = wl.config3()
    Wc = (oracle.margin(c) + wl.seeded_field(c, 21, 0.05)).astype(np.float32)
    gc, gf = hj.Grid.from_spec(c), hj.Grid.from_spec(f)
    gc.set_value(Wc)
    hj.prolong(gc, gf)
    Wf = gf.value()
    gc.close()
    gf.close()
    rng = np.random.default_rng(8)
    idx = rng.integers(0, 81, size=(4096, 4))
    X = [np.linspace(a, b, m) for a, b, m in zip(f.lo, f.hi, f.n)]
    pts = np.stack([X[d][idx[:, d]] for d in range(4)], axis=1)
    vo = oracle.query_value(c, Wc.astype(np.float64), pts)
    lo = np.array([oracle.margin_at(f, p) for p in pts])
    expect = np.minimum(vo, lo)
    got = Wf[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]]
    assert np.abs(got - expect).max() <= 2e-6 * np.abs(expect).max()


def test_config3_fine_grid_fixed_horizon_full_size(hj):
    """The adaptive update's fine grid at full size (81^4, 43 M nodes): a
    seeded coarse field on 31^4 is migrated to 81^4 and stepped 20 times
    (WENO5, monotone clamp, the shape-specialised kernels the bench times)
    from that start on both sides, at the oracle's dt; every node compared
    at the parity bar.  Both sides start from the same float32 coarse
    values."""
    c, f, _ = wl.config3()
    Wc = (oracle.margin(c) + wl.seeded_field(c, 31, 0.05)).astype(np.float32)
    dt = oracle.cfl_dt(f)
    gc, gf = hj.Grid.from_spec(c), hj.Grid.from_spec(f)
    gf.solve(hj.HJ_COLD, scheme=5, fixed_steps=1, dt=dt, clamp=1)
    assert hj.hj_jit_wait(120.0)
    gc.set_value(Wc)
    hj.prolong(gc, gf)
    st = gf.solve(hj.HJ_WARM, scheme=5, dt=dt, fixed_steps=20, clamp=1)
    Wg = gf.value()
    gc.close()
    gf.close()
    assert st["steps"] == 20
    W0 = oracle.prolong(c, Wc.astype(np.float64), f)
    Wo, _ = oracle.solve(f, scheme=5, dt=dt, fixed_steps=20, clamp=1, warm=W0)
    del W0
    assert_parity(Wg, Wo, f)


def read_x41_reference():
    """The stored FP64 oracle solve of the 41^4 x-subsystem at |d| <= 1.0
    (tests/golden/make_x41_reference.py): its step count, dt, max|W| and the
    sampled nodes with their values and far-from-zero-level flags."""
    import os
    import re
    path = os.path.join(os.path.dirname(__file__), "golden", "x41_b1.0_monotone_band_samples.txt")
    head = "".join(l for l in open(path) if l.startswith("#"))
    steps = int(re.search(r"steps=(\d+)", head).group(1))
    dt = float(re.search(r"dt=([0-9.eE+-]+)", head).group(1))
    m = re.search(r"max_abs_W=([0-9.eE+-]+)", head)
    a = np.loadtxt(path, comments="#")
    far = a[:, 5].astype(bool) if a.shape[1] > 5 else None
    return dict(steps=steps, dt=dt, max_abs=float(m.group(1)) if m else None,
                idx=a[:, :4].astype(np.int64), W=a[:, 4], far=far)


def test_x41_fixed_horizon_matches_stored_oracle_at_full_size(hj):
    """The bench's 4-D setting at full size (41^4, WENO5, monotone clamp):
    the GPU runs exactly the oracle's step count at the oracle's dt from the
    cold start, with the shape-specialised kernels the bench times, and is
    compared at the 4096 stored nodes with the parity bar: |dW| <= 1e-4
    max|W| and the sign the same at every stored node that lies more than one
    cell from the oracle's zero level set."""
    ref = read_x41_reference()
    assert ref["max_abs"] is not None and ref["far"] is not None
    spec = wl.quad_x4(41, 1.0)
    gpu_fixed(hj, spec, 5, 1, dt=ref["dt"], clamp=1)
    assert hj.hj_jit_wait(120.0) and hj.hj_jit_kernels() > 0
    Wg, st = gpu_fixed(hj, spec, 5, ref["steps"], dt=ref["dt"], clamp=1)
    assert st["steps"] == ref["steps"]
    i = ref["idx"]
    got = Wg[i[:, 0], i[:, 1], i[:, 2], i[:, 3]].astype(np.float64)
    err = np.abs(got - ref["W"]).max()
    assert err <= REL * ref["max_abs"], (err, ref["max_abs"])
    far = ref["far"] & (ref["W"] != 0)
    assert far.sum() > 2000
    agree = np.mean((got[far] >= 0) == (ref["W"][far] >= 0))
    assert agree >= SIGN_FRAC, agree
    # the GPU's own stop rule at the same dt stops within a few windows of the oracle's
    g = hj.Grid.from_spec(spec)
    stc = g.solve(hj.HJ_COLD, scheme=5, dt=ref["dt"], tol=1e-4, clamp=1, band=0.5,
                  max_steps=20000)
    g.close()
    per = int(np.ceil(0.1 / ref["dt"] - 1e-9))
    assert stc["converged"] and abs(stc["steps"] - ref["steps"]) <= 6 * per


@pytest.mark.parametrize("n", [17, 21])
def test_x4_converged_warm_update_parity_monotone_band(hj, n):
    """The bench's warm update in the 4-D setting (monotone clamp, band stop
    test), converged, against the oracle warm-started the same way: both sides
    solve b = 0 cold, then b = 0.5 warm from their own b = 0 result, with the
    oracle run to the GPU's stop step of each solve (the FP32 snapshots can
    move the stop a few windows), at the same dt.  Parity bar as above."""
    s0, s5 = wl.quad_x4(n, 0.0), wl.quad_x4(n, 0.5)
    dt0, dt5 = oracle.cfl_dt(s0), oracle.cfl_dt(s5)
    kw = dict(scheme=5, tol=1e-4, clamp=1, band=0.5)
    g = hj.Grid.from_spec(s0)
    st0 = g.solve(hj.HJ_COLD, dt=dt0, max_steps=60000, **kw)
    W0g = g.value()
    g.set_disturbance_bound([-0.5], [0.5])
    stw = g.solve(hj.HJ_WARM, dt=dt5, max_steps=60000, **kw)
    Wwg = g.value()
    g.close()
    assert st0["converged"] and stw["converged"]
    W0o, _ = oracle.solve(s0, scheme=5, dt=dt0, fixed_steps=st0["steps"], clamp=1)
    assert_parity(W0g, W0o, s0)
    Wwo, _ = oracle.solve(s5, scheme=5, dt=dt5, fixed_steps=stw["steps"], clamp=1, warm=W0o)
    assert_parity(Wwg, Wwo, s5)
    # the oracle's own stop rule from its own prior ends within a few windows
    _, sto = oracle.solve(s5, dt=dt5, max_steps=60000, warm=W0o, **kw)
    assert sto["converged"] and abs(sto["windows"] - stw["windows"]) <= 6


def test_x41_warm_and_cold_properties(hj):
    """A property test, not a parity claim: 41^4 cold solve with the 4-D
    workload setting (monotone clamp, band |W| <= 0.5 stop test): W <= l
    everywhere, W even under the point reflection of the symmetric
    x-subsystem, and the warm solve from the b = 0 fixed point gives nearly
    the same safe set.  Near the truncated v/theta/omega faces the monotone
    clamp keeps the downswings of the scheme's cycling, so the value there
    depends on the start (measured: up to 6e-2 at the faces, 2e-3 from eight
    cells in); values are compared from eight cells in.  Parity of each of
    the two solves against the oracle is the two tests above."""
    s0, s5 = wl.config1(b=0.0), wl.config1(b=0.5)
    g = hj.Grid.from_spec(s0)
    cap = dict(scheme=5, max_steps=100000, max_wall_ms=120000.0, band=0.5, clamp=1)
    st0 = g.solve(hj.HJ_COLD, **cap)
    assert st0["converged"]
    g.set_disturbance_bound([-0.5], [0.5])
    stw = g.solve(hj.HJ_WARM, **cap)
    Ww = g.value()
    stc = g.solve(hj.HJ_COLD, **cap)
    Wc = g.value()
    g.close()
    assert stw["converged"] and stc["converged"]
    l = oracle.margin(s5).astype(np.float32)
    assert np.all(Wc <= l)
    band = np.abs(Wc) <= 0.5
    assert np.abs(Wc - Wc[::-1, ::-1, ::-1, ::-1])[band].max() <= 1e-4 * np.abs(Wc).max()
    assert np.mean((Ww >= 0) == (Wc >= 0)) >= 0.999
    n = Wc.shape[0]
    I = np.indices(Wc.shape)
    face = np.min(np.stack([np.minimum(I[a], n - 1 - I[a]) for a in (1, 2, 3)]), axis=0)
    inner = band & (face >= 8)
    assert np.abs(Ww - Wc)[inner].max() <= 1e-3 * np.abs(Wc).max()


# ------------------------------------------------------------ edges

def test_argument_errors(hj):
    with pytest.raises(hj.HJError) as e:
        hj.hj_grid_create([2, 5], [0, 0], [1, 1])
    assert e.value.status == hj.HJ_ERR_ARG
    with pytest.raises(hj.HJError):
        hj.hj_grid_create([5], [1.0], [0.0])
    with pytest.raises(hj.HJError):
        hj.hj_grid_create([2000, 2000, 1000], [0, 0, 0], [1, 1, 1])  # >= 2^31 nodes
    g = hj.Grid([5, 5], [0, 0], [1, 1])
    rc, _ = hj.hj_solve(g.handle, 0, hj.make_opts(), raise_on_error=False)
    assert rc == hj.HJ_ERR_STATE
    hj.hj_set_dynamics(g.handle, "drift", [])
    hj.hj_set_constraint(g.handle, [0.2, -np.inf], [0.8, np.inf])
    rc, _ = hj.hj_solve(g.handle, 0, hj.make_opts(), raise_on_error=False)
    assert rc == hj.HJ_ERR_STATE  # disturbance not set
    hj.hj_set_disturbance_bound(g.handle, [-0.1, -0.1], [0.1, 0.1])
    rc, _ = hj.hj_solve(g.handle, 1, hj.make_opts(), raise_on_error=False)
    assert rc == hj.HJ_ERR_STATE  # warm without a prior
    with pytest.raises(hj.HJError):
        hj.hj_set_dynamics(g.handle, "quad_x4", list(wl.X4_PARAMS))  # wrong ndim
    g.close()


def test_step_cap_returns_not_converged_with_valid_tube(hj):
    spec = wl.quad_z(61, 0.5)
    g = hj.Grid.from_spec(spec)
    st = g.solve(hj.HJ_COLD, scheme=2, tol=1e-9, max_steps=17)
    assert st["status"] == hj.HJ_ERR_NOT_CONVERGED and st["steps"] == 17
    Wg = g.value()
    g.close()
    Wo, _ = oracle.solve(spec, scheme=2, dt=st["dt"], fixed_steps=17)
    assert_parity(Wg, Wo, spec)


def test_no_motion_converges_immediately(hj):
    spec = wl.drift((9, 9), 1.0, 0.0, wl.CON_BOX, r=0.5)
    g = hj.Grid.from_spec(spec)
    st = g.solve(hj.HJ_COLD, scheme=5)
    W = g.value()
    g.close()
    assert st["converged"] and st["steps"] == 0
    assert np.allclose(W, oracle.margin(spec), atol=1e-6)


def test_graph_and_direct_launch_agree(hj):
    spec = wl.quad_z(81, 0.5)
    out = []
    for graph in (True, False):
        g = hj.Grid.from_spec(spec)
        st = g.solve(hj.HJ_COLD, scheme=5, tol=1e-4, use_graph=graph)
        out.append((g.value(), st["steps"]))
        g.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


def test_device_pointer_io_and_stream(hj):
    import torch
    spec = wl.quad_z(41, 0.5)
    s = torch.cuda.Stream()
    g = hj.Grid.from_spec(spec, stream=s)
    t = torch.full((41 * 41,), 0.25, device="cuda", dtype=torch.float32)
    g.set_value(t)
    out = torch.empty_like(t)
    g.value_into(out)
    assert torch.equal(out, t)
    st = g.solve(hj.HJ_WARM, scheme=2, fixed_steps=3)
    g.value_into(out)
    torch.cuda.synchronize()
    W = out.cpu().numpy().reshape(41, 41)
    g.close()
    prior = np.full((41, 41), 0.25)
    Wo, _ = oracle.solve(spec, scheme=2, dt=st["dt"], fixed_steps=3, warm=prior)
    assert_parity(W, Wo, spec)


def test_kernel_launch_counter_moves(hj):
    before = hj.hj_kernel_launches()
    spec = wl.quad_z(21, 0.5)
    g = hj.Grid.from_spec(spec)
    g.solve(hj.HJ_COLD, scheme=2, fixed_steps=4)
    g.close()
    assert hj.hj_kernel_launches() - before >= 12


def test_autotune_keeps_value_and_results(hj):
    """The launch-shape autotuner only changes how the stage kernels map onto
    the GPU (flat block size or row tiles): W is left as it was, and solves
    after tuning give bit-identical results."""
    spec = wl.quad_x4(23, 0.5)
    g = hj.Grid.from_spec(spec)
    g.solve(hj.HJ_COLD, scheme=5, fixed_steps=3)
    before = g.value()
    t = hj.hj_autotune(g.handle, hj.HJ_WENO5)
    assert t in (128, 256, 512)
    threads, rows = g.launch_shape()
    assert threads == t and rows >= 0
    assert np.array_equal(g.value(), before)
    st1 = g.solve(hj.HJ_COLD, scheme=5, fixed_steps=7)
    W1 = g.value()
    g.close()
    g2 = hj.Grid.from_spec(spec)
    g2.solve(hj.HJ_COLD, scheme=5, fixed_steps=7, autotune=True)
    W2 = g2.value()
    g2.close()
    assert np.array_equal(W1, W2)
    dt = oracle.cfl_dt(spec)
    Wo, _ = oracle.solve(spec, scheme=5, dt=st1["dt"], fixed_steps=7)
    assert_parity(W1, Wo, spec)


def test_shape_specialised_kernels_match_precompiled_bitwise(hj):
    """Grids of >= 2^19 nodes run stage kernels compiled at run time with the
    grid shape as constants: the same values as the precompiled kernels,
    bit for bit, on direct launches and inside captured graphs."""
    cases = [(wl.quad_x4(33, 0.5), 5), (wl.quad_z(1025, 0.5), 2)]
    before = hj.hj_jit_kernels()
    out = {}
    try:
        for jit in (True, False):
            hj.hj_set_jit(jit)
            for spec, scheme in cases:
                g = hj.Grid.from_spec(spec)
                # the first launch starts the background compile; wait for it
                g.solve(hj.HJ_COLD, scheme=scheme, fixed_steps=1, use_graph=False)
                assert hj.hj_jit_wait(120.0)
                g.solve(hj.HJ_COLD, scheme=scheme, fixed_steps=6, use_graph=False)
                Wd = g.value()
                st = g.solve(hj.HJ_COLD, scheme=scheme, tol=1e-2, max_steps=400)
                Wg = g.value()
                g.close()
                out[(jit, spec.name)] = (Wd, Wg, st["steps"])
    finally:
        hj.hj_set_jit(True)
    assert hj.hj_jit_kernels() > before
    for spec, _ in cases:
        a, b = out[(True, spec.name)], out[(False, spec.name)]
        assert a[2] == b[2]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _run_shape(hj, spec, scheme, threads, rows, **kw):
    g = hj.Grid.from_spec(spec)
    g.set_launch_shape(threads, rows)
    assert g.launch_shape() == (threads, rows)
    g.solve(hj.HJ_COLD, scheme=scheme, fixed_steps=7, **kw)
    Wf = g.value()
    st = g.solve(hj.HJ_COLD, scheme=scheme, tol=1e-3, max_steps=300, **kw)
    Wc = g.value()
    g.close()
    return Wf, Wc, st


@pytest.mark.parametrize("name,spec,scheme,rows", [
    ("x4-ragged-weno5", wl.drift((13, 15, 9, 19), 1.0, 0.5), 5, (1, 5, 15, 53)),
    ("x4-weno5", wl.quad_x4(13, 0.5), 5, (1, 7, 13)),
    ("z-eno2", wl.quad_z(57, 0.5), 2, (1, 4, 17)),
    ("z-weno5", wl.quad_z(83, 0.5), 5, (1, 3, 12)),
    ("drift3-eno2", wl.drift((9, 11, 13), 1.0, 0.4), 2, (1, 9, 78)),
    ("drift1-weno5", wl.drift((300,), 1.0, 0.3), 5, (1,)),
    ("drift2-first", wl.drift((40, 31), 1.0, 0.3), 1, (2, 33)),
], ids=lambda v: v if isinstance(v, str) else "")
def test_row_tiles_match_flat_mapping_bitwise(hj, name, spec, scheme, rows):
    """Row tiles (lines of the fastest axis staged in shared memory with
    their ghost values) compute the same values as the flat one-node-per-
    thread mapping, bit for bit: fixed steps, and a converged solve (the
    window residual is reduced per block) with the same step count; for
    every line count, including tiles whose last one is short, and against
    the oracle."""
    Wf0, Wc0, st0 = _run_shape(hj, spec, scheme, 256, 0)
    for r in rows:
        Wf, Wc, st = _run_shape(hj, spec, scheme, 256, r)
        assert np.array_equal(Wf, Wf0), (name, r)
        assert np.array_equal(Wc, Wc0) and st["steps"] == st0["steps"], (name, r)
    dt = oracle.cfl_dt(spec)
    g = hj.Grid.from_spec(spec)
    g.set_launch_shape(256, rows[-1])
    g.solve(hj.HJ_COLD, scheme=scheme, dt=dt, fixed_steps=7)
    Wo, _ = oracle.solve(spec, scheme=scheme, dt=dt, fixed_steps=7)
    assert_parity(g.value(), Wo, spec)
    g.close()


def test_row_tiles_reject_shapes_that_do_not_fit(hj):
    g = hj.Grid.from_spec(wl.quad_x4(41, 0.5))
    with pytest.raises(hj.HJError):
        g.set_launch_shape(256, 25)  # 1025 nodes per tile
    with pytest.raises(hj.HJError):
        g.set_launch_shape(300, 0)
    g.set_launch_shape(256, 24)
    g.close()


def test_specialised_row_tiles_match_flat_bitwise(hj):
    """Row tiles compiled at run time for a grid of >= 2^19 nodes, on direct
    launches and inside captured graphs: the same values as the precompiled
    flat kernels, bit for bit."""
    spec = wl.quad_x4(33, 0.5)
    out = {}
    try:
        for jit, rows in ((False, 0), (True, 7), (True, 31)):
            hj.hj_set_jit(jit)
            g = hj.Grid.from_spec(spec)
            g.set_launch_shape(256, rows)
            g.solve(hj.HJ_COLD, scheme=5, fixed_steps=1, use_graph=False)
            assert hj.hj_jit_wait(120.0)
            g.solve(hj.HJ_COLD, scheme=5, fixed_steps=6, use_graph=False)
            Wd = g.value()
            st = g.solve(hj.HJ_COLD, scheme=5, tol=1e-2, max_steps=400)
            out[(jit, rows)] = (Wd, g.value(), st["steps"])
            g.close()
    finally:
        hj.hj_set_jit(True)
    ref = out[(False, 0)]
    for k, v in out.items():
        assert v[2] == ref[2] and np.array_equal(v[0], ref[0]) and np.array_equal(v[1], ref[1]), k


def test_exit_with_a_compile_running_is_clean(hj):
    """A process that exits while a shape-specialised compile still runs
    (it waits for it at exit) ends with status 0."""
    import subprocess
    import sys
    code = ("from paper_2101_05916_gb300 import hj, workloads as wl\n"
            "g = hj.Grid.from_spec(wl.quad_x4(35, 0.5))\n"
            "g.solve(hj.HJ_COLD, scheme=5, fixed_steps=1, use_graph=False)\n"
            "print('pending', hj.hj_jit_pending())\n")
    root = __file__.rsplit("/tests/", 1)[0]
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "pending" in r.stdout
