"""Seeded synthetic workloads for the HJ safe-set solve.

This module only *describes* inputs: grid boxes and sizes, model constants,
disturbance intervals, constraint boxes and the serving request trace.  It
holds none of the solver's arithmetic, so both the CUDA path and the FP64
oracle can take their inputs from here without sharing any computation.

Model constants follow the paper's near-hover quadcopter (Sec. IV, Eq. 3:
d0 = 10, d1 = 8, n0 = 10) and 2-D vertical quadcopter (Sec. V-A), in the
numeric form of the five benchmark configurations:

* z (2-D):  dz/dt = vz, dvz/dt = 0.91 u - 9.81 + d, u in [0, 19.62]
* x (4-D):  dx/dt = vx + d, dvx/dt = 9.81 tan(thx), dthx/dt = -8 thx + wx,
            dwx/dt = -10 thx + 10 u, u in [-pi/9, pi/9]
* y (4-D):  the same model as x with its own constraint box.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

INF = math.inf

# model names understood by both the library binding and the oracle binding
DRIFT = "drift"
QUAD_Z = "quad_z"
QUAD_X4 = "quad_x4"

CON_BOX = "box"            # safe inside an axis-aligned box
CON_BALL_OUT = "ball_out"  # safe outside a ball

# z: (kT, g, u_lo, u_hi)
Z_PARAMS = (0.91, 9.81, 0.0, 19.62)
# x / y: (g, d1, d0, n0, u_lo, u_hi, disturbance axis)
X4_PARAMS = (9.81, 8.0, 10.0, 10.0, -math.pi / 9.0, math.pi / 9.0, 0.0)


@dataclasses.dataclass
class ProblemSpec:
    """One subsystem grid problem: grid, dynamics, disturbance box, constraint."""

    name: str
    n: Tuple[int, ...]
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    model: str
    params: Tuple[float, ...]
    d_lo: Tuple[float, ...]
    d_hi: Tuple[float, ...]
    con_kind: str
    con_a: Tuple[float, ...]   # box lo, or ball centre
    con_b: Tuple[float, ...]   # box hi, or (radius,)

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def npts(self) -> int:
        return int(np.prod(self.n))

    def h(self) -> Tuple[float, ...]:
        return tuple((b - a) / (m - 1) for a, b, m in zip(self.lo, self.hi, self.n))

    def coords(self) -> List[np.ndarray]:
        return [np.linspace(a, b, m) for a, b, m in zip(self.lo, self.hi, self.n)]

    def with_bound(self, b: float) -> "ProblemSpec":
        """Same problem with the symmetric disturbance interval [-b, b] on every input."""
        k = len(self.d_lo)
        return dataclasses.replace(self, d_lo=(-b,) * k, d_hi=(b,) * k)

    def with_grid(self, n: Sequence[int]) -> "ProblemSpec":
        return dataclasses.replace(self, n=tuple(int(v) for v in n))

    def key(self) -> Tuple:
        """Identity of (model, grid, constraint) used for warm-start residency."""
        return (self.model, self.params, self.n, self.lo, self.hi, self.con_kind,
                self.con_a, self.con_b)


def quad_z(n: int = 101, b: float = 0.5, z_box=(0.5, 2.5), name: str = "z") -> ProblemSpec:
    """2-D vertical quadcopter subsystem on z in [0, 3], vz in [-3, 3]."""
    return ProblemSpec(name=name, n=(n, n), lo=(0.0, -3.0), hi=(3.0, 3.0), model=QUAD_Z,
                       params=Z_PARAMS, d_lo=(-b,), d_hi=(b,), con_kind=CON_BOX,
                       con_a=(z_box[0], -INF), con_b=(z_box[1], INF))


def quad_x4(n: int = 41, b: float = 0.5, half_width: float = 4.0, name: str = "x",
            shift: float = 0.0) -> ProblemSpec:
    """4-D x (or y) subsystem over [-5,5] x [-2,2] x [-0.35,0.35] x [-1.5,1.5]
    with constraint |p - shift| <= half_width."""
    return ProblemSpec(name=name, n=(n,) * 4, lo=(-5.0, -2.0, -0.35, -1.5),
                       hi=(5.0, 2.0, 0.35, 1.5), model=QUAD_X4, params=X4_PARAMS,
                       d_lo=(-b,), d_hi=(b,), con_kind=CON_BOX,
                       con_a=(shift - half_width, -INF, -INF, -INF),
                       con_b=(shift + half_width, INF, INF, INF))


def drift(n: Sequence[int], half: float, b: float, con_kind: str = CON_BOX,
          r: float = 1.0) -> ProblemSpec:
    """dx/dt = d with |d_i| <= b, on [-half, half]^D; box |x_i| <= r or ball |x| >= r."""
    D = len(n)
    if con_kind == CON_BOX:
        ca, cb = (-r,) * D, (r,) * D
    else:
        ca, cb = (0.0,) * D, (r,)
    return ProblemSpec(name=f"drift{D}", n=tuple(n), lo=(-half,) * D, hi=(half,) * D,
                       model=DRIFT, params=(), d_lo=(-b,) * D, d_hi=(b,) * D,
                       con_kind=con_kind, con_a=ca, con_b=cb)


def demo10d_x(n: int = 31, b: float = 0.5, name: str = "x") -> ProblemSpec:
    """x (or y) subsystem under the 10-D demo's constraint boxes (Sec. V):
    |p| <= 2.5, |v| <= 3.5 and |theta| <= pi/8 together, on a grid that holds
    the box with a margin: [-3.5,3.5] x [-4.5,4.5] x [-0.5,0.5] x [-2,2]."""
    t = math.pi / 8.0
    return ProblemSpec(name=name, n=(n,) * 4, lo=(-3.5, -4.5, -0.5, -2.0),
                       hi=(3.5, 4.5, 0.5, 2.0), model=QUAD_X4, params=X4_PARAMS,
                       d_lo=(-b,), d_hi=(b,), con_kind=CON_BOX,
                       con_a=(-2.5, -3.5, -t, -INF), con_b=(2.5, 3.5, t, INF))


def demo10d_z(n: int = 101, b: float = 0.5) -> ProblemSpec:
    """z subsystem under the 10-D demo's boxes (Sec. V): z in [0.35, 2.8] and
    |v_z| <= 3.5, on [0, 3.2] x [-4.5, 4.5]."""
    return ProblemSpec(name="z", n=(n, n), lo=(0.0, -4.5), hi=(3.2, 4.5), model=QUAD_Z,
                       params=Z_PARAMS, d_lo=(-b,), d_hi=(b,), con_kind=CON_BOX,
                       con_a=(0.35, -3.5), con_b=(2.8, 3.5))


def two_band_margin(spec: ProblemSpec, bands: Sequence[Tuple[float, float]],
                    axis: int = 0) -> np.ndarray:
    """Margin l of a non-convex safe set: the union of slabs lo <= x_axis <= hi
    (distance to the nearest face of the slab the node lies in, else minus the
    distance to the nearest slab), on every node of the grid."""
    xs = np.meshgrid(*spec.coords(), indexing="ij")[axis]
    return np.max([np.minimum(xs - lo, hi - xs) for lo, hi in bands], axis=0)


# The 10-D near-hover quadcopter (Sec. IV): state (p_x, v_x, th_x, w_x, p_y,
# v_y, th_y, w_y, p_z, v_z), inputs (u_x, u_y, T_z), decomposed into the x,
# y and z subsystems.  State indices of each subsystem's axes, and the input
# each subsystem drives.
QUAD10D_AXES = ((0, 1, 2, 3), (4, 5, 6, 7), (8, 9))
QUAD10D_CTRL = (0, 1, 2)


def quad10d_states(specs: Sequence[ProblemSpec], count: int, seed: int = 7,
                   inset: float = 0.02) -> np.ndarray:
    """Seeded full 10-D states, uniform inside every subsystem grid box
    (shrunk by `inset` of each axis length), for filter queries."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((count, 10))
    for spec, axes in zip(specs, QUAD10D_AXES):
        for d, a in enumerate(axes):
            w = spec.hi[d] - spec.lo[d]
            out[:, a] = rng.uniform(spec.lo[d] + inset * w, spec.hi[d] - inset * w, count)
    return out


# ---------------------------------------------------------------- configs

def config0() -> ProblemSpec:
    """Plain cold 2-D z solve, 101 x 101, wind |d| <= 0.5, ENO2."""
    return quad_z(101, 0.5)


def config1(n: int = 41, b: float = 0.5) -> ProblemSpec:
    """4-D x subsystem, 41^4, |x| <= 4, |d| <= 0.5, WENO5 (cold vs warm)."""
    return quad_x4(n, b)


def config2(n4: int = 61, n2: int = 201) -> List[ProblemSpec]:
    """Decomposed 10-D quadcopter as one batch: x and y at 61^4, z at 201^2.
    y uses its own constraint |y| <= 3.5 so that the batch holds two distinct grids."""
    return [quad_x4(n4, 0.0, 4.0, "x"), quad_x4(n4, 0.0, 3.5, "y"), quad_z(n2, 0.0)]


CONFIG2_BOUNDS = (0.0, 0.5, 1.0, 1.5)


def config3() -> Tuple[ProblemSpec, ProblemSpec, ProblemSpec]:
    """Adaptive grid on x: coarse 31^4, fine 81^4, reference 41^4; wind 1.0."""
    return quad_x4(31, 1.0), quad_x4(81, 1.0), quad_x4(41, 1.0)


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    spec: ProblemSpec
    scheme: int


def serving_trace(count: int = 256, rate_hz: float = 20.0, seed: int = 20210115,
                  n2: Tuple[int, int] = (101, 401), n4: Tuple[int, int] = (31, 71),
                  bmax: float = 1.5, shift: float = 0.2) -> List[Request]:
    """Poisson arrivals of safety-update requests of random subsystem type and size.

    Subsystem type uniform over {z, x, y}; grid points per axis uniform in
    n2 (2-D) or n4 (4-D); wind bound uniform in [0, bmax]; constraint box
    translated by s * width with s uniform in [-shift, shift].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate_hz)
        kind = int(rng.integers(0, 3))
        b = float(rng.uniform(0.0, bmax))
        s = float(rng.uniform(-shift, shift))
        if kind == 2:
            n = int(rng.integers(n2[0], n2[1] + 1))
            w = 2.0
            spec = quad_z(n, b, (0.5 + s * w, 2.5 + s * w), name="z")
            scheme = 2
        else:
            n = int(rng.integers(n4[0], n4[1] + 1))
            hw = 4.0 if kind == 0 else 3.5
            spec = quad_x4(n, b, hw, "x" if kind == 0 else "y", shift=s * 2 * hw)
            scheme = 5
        out.append(Request(rid, t, spec, scheme))
    return out


def wind_field(spec: ProblemSpec, base: float, bump: float, axis: int, centre: float,
               width: float) -> Tuple[np.ndarray, np.ndarray]:
    """A GP-like state-dependent wind interval (Sec. II-C, Sec. V-A: the fan's
    wind is strongest near one place and fades away from it):
    |d| <= base + bump * exp(-((x_axis - centre) / width)^2) at every node.
    Returns (d_lo, d_hi), each of shape (nd,) + grid shape."""
    xs = np.meshgrid(*spec.coords(), indexing="ij")[axis]
    b = base + bump * np.exp(-((xs - centre) / width) ** 2)
    nd = len(spec.d_lo)
    hi = np.broadcast_to(b, (nd,) + tuple(spec.n)).astype(np.float64).copy()
    return -hi, hi


def seeded_field(spec: ProblemSpec, seed: int, scale: float = 1.0) -> np.ndarray:
    """A reproducible random field on the grid (for layout and edge tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (scale * rng.standard_normal(spec.n)).astype(np.float64)
