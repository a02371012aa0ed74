"""Writes tests/golden/x41_b1.0_monotone_band_samples.txt.

The FP64 oracle's converged value of the 4-D x-subsystem on a 41^4 grid at
wind bound 1.0 (WENO5, TVD-RK3, CFL 0.5, monotone clamp, stop at a window
change below 1e-4 on the band |W| <= 0.5), sampled at 4096 seeded nodes.

The header records the oracle's step count and dt, so that a run of exactly
that many steps at that dt is a fixed-horizon comparison at full size, and
max|W| over the whole grid, the scale of the parity tolerance.  Each sample
row carries a flag `far`: 1 when no neighbour of the node along any axis has
the other sign of W (the node lies more than one cell from the zero level
set), which is where the sign test applies.

It is also the reference for the coarse-to-fine error report: a 81^4 result
restricted to every second node lands on this 41^4 grid.  Calls only the
oracle; takes tens of minutes on a few cores.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2101_05916_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "x41_b1.0_monotone_band_samples.txt")


def sample_indices(n=41, count=4096, seed=41):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, n, size=(count, 4))


def far_from_zero_level(W):
    """True where every axis neighbour has the node's sign (W >= 0 or < 0)."""
    pos = W >= 0
    near = np.zeros(W.shape, dtype=bool)
    for ax in range(W.ndim):
        lo = [slice(None)] * W.ndim
        hi = [slice(None)] * W.ndim
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        diff = pos[tuple(lo)] != pos[tuple(hi)]
        near[tuple(lo)] |= diff
        near[tuple(hi)] |= diff
    return ~near & (W != 0)


def main(out=OUT):
    spec = wl.quad_x4(41, 1.0)
    t0 = time.time()
    W, st = oracle.solve(spec, scheme=5, tol=1e-4, clamp=1, band=0.5, max_steps=200000)
    far = far_from_zero_level(W)
    idx = sample_indices()
    with open(out, "w") as f:
        f.write("# oracle: 4-D x subsystem 41^4, |d|<=1.0, WENO5, TVD-RK3, CFL 0.5, monotone clamp,\n")
        f.write("# band 0.5 stop test at 1e-4; steps=%d dt=%.17g converged=%d safe_fraction=%.6f "
                "seconds=%.0f\n" % (st["steps"], st["dt"], st["converged"], float(np.mean(W >= 0)),
                                    time.time() - t0))
        f.write("# max_abs_W=%.17g\n" % float(np.abs(W).max()))
        f.write("# i0 i1 i2 i3 W far\n")
        for i in idx:
            t = tuple(i)
            f.write("%d %d %d %d %.17e %d\n" % (i[0], i[1], i[2], i[3], W[t], int(far[t])))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else OUT)
