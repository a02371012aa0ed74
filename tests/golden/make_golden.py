"""Writes the stored oracle outputs under tests/golden/.

Calls only the FP64 oracle (oracle/) on the seeded workloads; nothing here
touches the CUDA library.  Re-run only when the oracle's arithmetic changes,
and say in the commit which passage or reading of the paper justifies it.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2101_05916_gb300 import workloads as wl  # noqa: E402


def write(name, spec, W, stats, header):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        f.write("# %s\n" % header)
        f.write("# grid n=%s lo=%s hi=%s steps=%d dt=%.17g\n"
                % (list(spec.n), list(spec.lo), list(spec.hi), stats["steps"], stats["dt"]))
        for v in W.ravel():
            f.write("%.17e\n" % v)


def main():
    s = wl.quad_z(41, 0.5)
    W, st = oracle.solve(s, scheme=2, tol=1e-9)
    write("z41_eno2_b0.5_converged.txt", s, W, st,
          "oracle: 2-D z subsystem, 41x41, |d|<=0.5, ENO2, TVD-RK3, CFL 0.5, converged to 1e-9")
    x = wl.quad_x4(9, 0.5)
    W, st = oracle.solve(x, scheme=5, fixed_steps=5)
    write("x9_weno5_b0.5_5steps.txt", x, W, st,
          "oracle: 4-D x subsystem, 9^4, |d|<=0.5, WENO5, TVD-RK3, CFL 0.5, 5 steps")


if __name__ == "__main__":
    main()
