"""ctypes binding of the FP64 CPU oracle (hj_oracle.c) plus a pure-Python
brute-force game-tree solver used to pin it.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the cpu_baseline / reference legs of bench.py.  The CUDA product path never
imports this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hj_oracle.c")
_LIB = os.path.join(_HERE, "libhj_oracle.so")

MAXD = 6
MAXIN = 6
_MODEL = {"drift": 0, "quad_z": 1, "quad_x4": 2}
_CON = {"box": 0, "ball_out": 1}
_CON_FIELD = 2


class _Problem(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_long * MAXD),
                ("lo", ctypes.c_double * MAXD), ("hi", ctypes.c_double * MAXD),
                ("model", ctypes.c_int), ("params", ctypes.c_double * 8),
                ("nd", ctypes.c_int), ("d_lo", ctypes.c_double * MAXIN),
                ("d_hi", ctypes.c_double * MAXIN), ("con_kind", ctypes.c_int),
                ("con_a", ctypes.c_double * MAXD), ("con_b", ctypes.c_double * MAXD),
                ("dflo", ctypes.c_void_p), ("dfhi", ctypes.c_void_p),
                ("lfield", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("cfl", ctypes.c_double), ("dt", ctypes.c_double),
                ("tol", ctypes.c_double), ("check_dt", ctypes.c_double),
                ("max_steps", ctypes.c_long), ("fixed_steps", ctypes.c_long),
                ("clamp", ctypes.c_int), ("warm", ctypes.c_int), ("band", ctypes.c_double),
                ("band_margin", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_long), ("t", ctypes.c_double),
                ("residual", ctypes.c_double), ("dt", ctypes.c_double),
                ("converged", ctypes.c_int), ("windows", ctypes.c_long)]


def build(force: bool = False) -> str:
    """Compile hj_oracle.c into a shared library next to it (gcc, OpenMP).
    HJ_ORACLE_LIB names an already built library to load instead (the
    mutation check of mutation_check.py runs the pins against modified
    copies that way)."""
    override = os.environ.get("HJ_ORACLE_LIB")
    if override:
        return override
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        _lib.or_solve.argtypes = [P(_Problem), P(_Opts), P(d), P(_Stats)]
        _lib.or_solve.restype = ctypes.c_int
        _lib.or_alpha.argtypes = [P(_Problem), P(d)]
        _lib.or_cfl_dt.argtypes = [P(_Problem), d, P(d)]
        _lib.or_cfl_dt.restype = d
        _lib.or_hamiltonian.argtypes = [P(_Problem), P(d), P(d)]
        _lib.or_hamiltonian.restype = d
        _lib.or_margin.argtypes = [P(_Problem), P(d)]
        _lib.or_margin.restype = d
        _lib.or_fill_margin.argtypes = [P(_Problem), P(d)]
        _lib.or_line_slopes.argtypes = [P(d), ctypes.c_long, d, ctypes.c_int, P(d), P(d)]
        _lib.or_rhs.argtypes = [P(_Problem), ctypes.c_int, P(d), P(d)]
        _lib.or_prolong.argtypes = [P(_Problem), P(d), P(_Problem), P(d)]
        _lib.or_prolong.restype = ctypes.c_int
        _lib.or_query_value.argtypes = [P(_Problem), P(d), ctypes.c_long, P(d), P(d)]
        _lib.or_query_value.restype = ctypes.c_int
        _lib.or_query_gradient.argtypes = [P(_Problem), P(d), ctypes.c_long, P(d), P(d)]
        _lib.or_query_gradient.restype = ctypes.c_int
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_set_num_threads.argtypes = [ctypes.c_int]
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _problem(spec, dfield=None, lfield=None) -> _Problem:
    """ctypes problem for a spec; dfield = (d_lo, d_hi) arrays of shape
    (nd,) + grid shape for a state-dependent disturbance box; lfield = the
    margin l on the grid, replacing the spec's analytic constraint (arrays
    kept alive by the caller for the duration of the call)."""
    p = _Problem()
    if dfield is not None:
        p.dflo = dfield[0].ctypes.data
        p.dfhi = dfield[1].ctypes.data
    p.ndim = spec.ndim
    for i in range(spec.ndim):
        p.n[i] = spec.n[i]
        p.lo[i] = spec.lo[i]
        p.hi[i] = spec.hi[i]
    p.model = _MODEL[spec.model]
    for i, v in enumerate(spec.params):
        p.params[i] = v
    p.nd = len(spec.d_lo)
    for i in range(p.nd):
        p.d_lo[i] = spec.d_lo[i]
        p.d_hi[i] = spec.d_hi[i]
    p.con_kind = _CON[spec.con_kind]
    for i, v in enumerate(spec.con_a):
        p.con_a[i] = v
    for i, v in enumerate(spec.con_b):
        p.con_b[i] = v
    if lfield is not None:
        p.con_kind = _CON_FIELD
        p.lfield = lfield.ctypes.data
    return p


def _lf(spec, lfield):
    if lfield is None:
        return None
    a = np.ascontiguousarray(lfield, dtype=np.float64)
    if a.size != spec.npts:
        raise ValueError("lfield must hold one value per node")
    return a


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(k: int) -> None:
    lib().or_set_num_threads(int(k))


def solve(spec, scheme: int = 5, cfl: float = 0.5, dt: float = 0.0, tol: float = 1e-4,
          check_dt: float = 0.1, max_steps: int = 0, fixed_steps: int = 0,
          clamp: int = 0, warm: Optional[np.ndarray] = None,
          band: float = 0.0, band_margin: int = 0,
          dfield: Optional[Tuple[np.ndarray, np.ndarray]] = None,
          lfield: Optional[np.ndarray] = None) -> Tuple[np.ndarray, Dict]:
    """Run the oracle solve; returns (W on the grid, stats).  dfield: optional
    state-dependent disturbance box (d_lo, d_hi), each (nd,) + grid shape.
    lfield: optional constraint given as its margin l on the grid."""
    dfield = _field(dfield)
    lfield = _lf(spec, lfield)
    W = np.zeros(spec.n, dtype=np.float64)
    if warm is not None:
        W[...] = warm
    o = _Opts(scheme=scheme, cfl=cfl, dt=dt, tol=tol, check_dt=check_dt, max_steps=max_steps,
              fixed_steps=fixed_steps, clamp=clamp, warm=1 if warm is not None else 0,
              band=band, band_margin=band_margin)
    st = _Stats()
    pr = _problem(spec, dfield, lfield)
    rc = lib().or_solve(ctypes.byref(pr), ctypes.byref(o), _dp(W), ctypes.byref(st))
    if rc < 0:
        raise ValueError("oracle rejected the problem")
    return W, dict(steps=st.steps, t=st.t, residual=st.residual, dt=st.dt,
                   converged=bool(st.converged), windows=st.windows, rc=rc)


def _field(dfield):
    if dfield is None:
        return None
    return (np.ascontiguousarray(dfield[0], dtype=np.float64),
            np.ascontiguousarray(dfield[1], dtype=np.float64))


def alpha(spec, dfield=None) -> np.ndarray:
    a = np.zeros(spec.ndim)
    dfield = _field(dfield)
    pr = _problem(spec, dfield)
    lib().or_alpha(ctypes.byref(pr), _dp(a))
    return a


def cfl_dt(spec, cfl: float = 0.5, dfield=None) -> float:
    a = alpha(spec, dfield)
    pr = _problem(spec)
    return lib().or_cfl_dt(ctypes.byref(pr), cfl, _dp(a))


def hamiltonian(spec, x: Sequence[float], p: Sequence[float]) -> float:
    xa = np.ascontiguousarray(x, dtype=np.float64)
    pa = np.ascontiguousarray(p, dtype=np.float64)
    pr = _problem(spec)
    return lib().or_hamiltonian(ctypes.byref(pr), _dp(xa), _dp(pa))


def margin(spec, lfield=None) -> np.ndarray:
    out = np.zeros(spec.n, dtype=np.float64)
    lfield = _lf(spec, lfield)
    pr = _problem(spec, None, lfield)
    lib().or_fill_margin(ctypes.byref(pr), _dp(out))
    return out


def margin_at(spec, x: Sequence[float]) -> float:
    xa = np.ascontiguousarray(x, dtype=np.float64)
    pr = _problem(spec)
    return lib().or_margin(ctypes.byref(pr), _dp(xa))


def line_slopes(w: np.ndarray, h: float, scheme: int) -> Tuple[np.ndarray, np.ndarray]:
    w = np.ascontiguousarray(w, dtype=np.float64)
    pm = np.zeros_like(w)
    pp = np.zeros_like(w)
    lib().or_line_slopes(_dp(w), w.size, h, scheme, _dp(pm), _dp(pp))
    return pm, pp


def rhs(spec, scheme: int, W: np.ndarray) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros_like(W)
    pr = _problem(spec)
    lib().or_rhs(ctypes.byref(pr), scheme, _dp(W), _dp(out))
    return out


def prolong(coarse, Wc: np.ndarray, fine, lfield_fine=None) -> np.ndarray:
    Wc = np.ascontiguousarray(Wc, dtype=np.float64)
    Wf = np.zeros(fine.n, dtype=np.float64)
    lfield_fine = _lf(fine, lfield_fine)
    pc, pf = _problem(coarse), _problem(fine, None, lfield_fine)
    if lib().or_prolong(ctypes.byref(pc), _dp(Wc), ctypes.byref(pf), _dp(Wf)) != 0:
        raise ValueError("fine grid not inside coarse grid")
    return Wf


def translate(src, Ws: np.ndarray, dst, shift: Sequence[float], lfield_dst=None) -> np.ndarray:
    """Translated prior: W_dst(x) = min(W_src(x - shift), l_dst(x)) by
    multilinear interpolation; l_dst(x) where x - shift leaves src's box."""
    Ws = np.ascontiguousarray(Ws, dtype=np.float64)
    X = np.stack([a.ravel() for a in np.meshgrid(*dst.coords(), indexing="ij")], axis=1)
    Y = X - np.asarray(shift, dtype=np.float64)[None, :]
    t = (Y - np.asarray(src.lo)[None, :]) / np.asarray(src.h())[None, :]
    inside = np.all((t >= -1e-9) & (t <= (np.asarray(src.n) - 1)[None, :] + 1e-9), axis=1)
    l = margin(dst, lfield_dst).ravel()
    out = l.copy()
    if inside.any():
        out[inside] = np.minimum(query_value(src, Ws, Y[inside]), l[inside])
    return out.reshape(dst.n)


def query_value(spec, W: np.ndarray, xs: np.ndarray) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    xs = np.ascontiguousarray(xs, dtype=np.float64).reshape(-1, spec.ndim)
    out = np.zeros(xs.shape[0])
    pr = _problem(spec)
    if lib().or_query_value(ctypes.byref(pr), _dp(W), xs.shape[0], _dp(xs), _dp(out)) != 0:
        raise ValueError("query point outside the grid")
    return out


def query_gradient(spec, W: np.ndarray, xs: np.ndarray) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    xs = np.ascontiguousarray(xs, dtype=np.float64).reshape(-1, spec.ndim)
    out = np.zeros_like(xs)
    pr = _problem(spec)
    if lib().or_query_gradient(ctypes.byref(pr), _dp(W), xs.shape[0], _dp(xs), _dp(out)) != 0:
        raise ValueError("query point outside the grid")
    return out


# ------------------------------------------------------------------ safety filter

def control_gain(spec) -> Tuple[np.ndarray, float, float]:
    """df/du of the subsystem's single input and its box, from the model
    definitions: z has dv/dt = kT u - g + d, x/y have dw/dt = -d0 th + n0 u.
    A drift has no input (gain 0)."""
    b = np.zeros(spec.ndim)
    if spec.model == "quad_z":
        b[1] = spec.params[0]
        return b, spec.params[2], spec.params[3]
    if spec.model == "quad_x4":
        b[3] = spec.params[3]
        return b, spec.params[4], spec.params[5]
    return b, 0.0, 0.0


def safety_filter(specs, Ws, axes, ctrl_index, states: np.ndarray, u_perf: np.ndarray,
                  level: float = 0.0):
    """Safe-learning switch over decomposed subsystems (Sec. II-A, II-B, III-A):
    W = min_k W_k; where W_k <= level the control of subsystem k becomes
    argmax_u min_d <grad W_k, f_k> (bang-bang; a tie keeps the performance
    control, clipped to the input box).  Returns (u, w, active mask)."""
    states = np.asarray(states, dtype=np.float64)
    u = np.array(u_perf, dtype=np.float64, copy=True)
    nq = states.shape[0]
    w = np.full(nq, np.inf)
    active = np.zeros(nq, dtype=np.int64)
    for k, (spec, W) in enumerate(zip(specs, Ws)):
        xs = states[:, list(axes[k][:spec.ndim])]
        wk = query_value(spec, W, xs)
        gk = query_gradient(spec, W, xs)
        w = np.minimum(w, wk)
        b, ulo, uhi = control_gain(spec)
        c = ctrl_index[k]
        if c < 0 or not b.any():
            continue
        s = gk @ b
        on = wk <= level
        us = np.where(s > 0, uhi, np.where(s < 0, ulo, np.clip(u[:, c], ulo, uhi)))
        u[on, c] = us[on]
        active[on] |= 1 << k
    return u, w, active


# ------------------------------------------------------------------ brute force

def _z_arc_extremes(z0, v0, a, tau):
    """Min and max of z(t) = z0 + v0 t + a t^2 / 2 over t in [0, tau] (arrays)."""
    z1 = z0 + v0 * tau + 0.5 * a * tau * tau
    lo = np.minimum(z0, z1)
    hi = np.maximum(z0, z1)
    ts = np.where(a != 0.0, -v0 / np.where(a != 0.0, a, 1.0), -1.0)
    inside = (ts > 0.0) & (ts < tau)
    zs = z0 + v0 * ts + 0.5 * a * ts * ts
    lo = np.where(inside, np.minimum(lo, zs), lo)
    hi = np.where(inside, np.maximum(hi, zs), hi)
    return lo, hi


def brute_force_z(z0: np.ndarray, v0: np.ndarray, horizon: float, intervals: int,
                  kT: float, g: float, u_set: Sequence[float], d_set: Sequence[float],
                  zlo: float, zhi: float, disturbance_last: bool) -> np.ndarray:
    """Value of the discrete game W = inf_d sup_u min_t l(z(t)) for the 2-D
    double integrator with piecewise-constant inputs drawn from finite sets.

    disturbance_last=True: in every interval the disturbance picks after
    seeing the control (max_u min_d per interval) -- the disturbance's
    information advantage, giving the lower bracket.  False: the control
    picks after the disturbance (min_d max_u), the upper bracket.
    The margin l(z) = min(z - zlo, zhi - z) is evaluated exactly along each
    arc via the arc's extreme heights (l is concave in z).
    """
    tau = horizon / intervals

    def margin_of(z):
        return np.minimum(z - zlo, zhi - z)

    def rec(z, v, m, depth):
        if depth == intervals:
            return m
        outs_u = []
        for u in u_set:
            outs_d = []
            for d in d_set:
                a = kT * u - g + d
                lo, hi = _z_arc_extremes(z, v, a, tau)
                m2 = np.minimum(m, np.minimum(margin_of(lo), margin_of(hi)))
                z2 = z + v * tau + 0.5 * a * tau * tau
                v2 = v + a * tau
                outs_d.append((u, d, z2, v2, m2))
            outs_u.append(outs_d)
        if disturbance_last:
            best = None
            for outs_d in outs_u:
                worst = None
                for (_, _, z2, v2, m2) in outs_d:
                    r = rec(z2, v2, m2, depth + 1)
                    worst = r if worst is None else np.minimum(worst, r)
                best = worst if best is None else np.maximum(best, worst)
            return best
        # control last: min over d of max over u
        worst = None
        for j in range(len(d_set)):
            best = None
            for outs_d in outs_u:
                (_, _, z2, v2, m2) = outs_d[j]
                r = rec(z2, v2, m2, depth + 1)
                best = r if best is None else np.maximum(best, r)
            worst = best if worst is None else np.minimum(worst, best)
        return worst

    z0 = np.asarray(z0, dtype=np.float64)
    v0 = np.asarray(v0, dtype=np.float64)
    return rec(z0, v0, margin_of(z0), 0)


def z_closed_form(z: np.ndarray, v: np.ndarray, kT: float, g: float, u_hi: float,
                  u_lo: float, b: float, zlo: float, zhi: float) -> np.ndarray:
    """Converged value of the 2-D double integrator against worst-case wind:
    the distance left to the nearer wall after braking at full authority."""
    a_up = kT * u_hi - g - b  # best upward acceleration under the worst wind
    a_dn = g - kT * u_lo - b  # best downward acceleration magnitude
    lo_side = z - zlo - np.where(v < 0.0, v * v / (2.0 * a_up), 0.0)
    hi_side = zhi - z - np.where(v > 0.0, v * v / (2.0 * a_dn), 0.0)
    return np.minimum(lo_side, hi_side)


__all__ = ["build", "lib", "solve", "alpha", "cfl_dt", "hamiltonian", "margin", "margin_at",
           "line_slopes", "rhs", "prolong", "query_value", "query_gradient", "brute_force_z",
           "z_closed_form", "num_threads", "set_num_threads", "control_gain", "safety_filter",
           "translate"]

