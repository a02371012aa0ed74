"""The end rule of the stage kernels' grid lines, checked on the host.

Ghost nodes continue a grid line linearly through its two outermost nodes
(the boundary reading of the method), so a one-sided difference that
reaches past an end equals the line's edge difference.  The kernels apply
that rule to the differences of a line (hjd::edge_diffs, hj_device.cuh)
rather than to its values.  This test compiles those helpers into a host
program and checks, for every node of lines of 3 to 12 nodes and stencil
radii 1 to 3, that the differences equal the ones the linear continuation
defines, bit for bit, whether the values beyond the ends are clamped copies
(the slower axes) or garbage (the fastest axis reads into the next row).
Runs on the CPU."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_05916_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include "hj_device.cuh"

template <int R>
static int check(int n) {
  float w[16];
  for (int j = 0; j < n; ++j) w[j] = (float)(3.0 * std::sin(1.7 * j + 0.3 * n) + 0.1 * j);
  for (int i = 0; i < n; ++i) {
    float vc[2 * R + 1], vg[2 * R + 1], Dc[2 * R], Dg[2 * R];
    for (int k = -R; k <= R; ++k) {
      int j = i + k;
      vc[k + R] = w[j < 0 ? 0 : (j > n - 1 ? n - 1 : j)];
      vg[k + R] = (j >= 0 && j < n) ? w[j] : NAN;
    }
    hjd::diffs_of<R>(vc, Dc);
    hjd::edge_diffs<R>(Dc, i, n);
    hjd::diffs_of<R>(vg, Dg);
    hjd::edge_diffs<R>(Dg, i, n);
    for (int k = 0; k < 2 * R; ++k) {
      int a = i + k - R;  // the slot spans nodes a and a + 1
      float want = (a + 1 <= 0) ? w[1] - w[0] : (a >= n - 1) ? w[n - 1] - w[n - 2] : w[a + 1] - w[a];
      if (!(Dc[k] == want) || !(Dg[k] == want)) {
        std::printf("MISMATCH R=%d n=%d i=%d k=%d want=%.9g clamped=%.9g garbage=%.9g\n", R, n, i,
                    k, want, Dc[k], Dg[k]);
        return 1;
      }
    }
  }
  return 0;
}

int main() {
  int bad = 0;
  for (int n = 3; n <= 12; ++n) bad |= check<1>(n) | check<2>(n) | check<3>(n);
  if (!bad) std::printf("OK\n");
  return bad;
}
"""


def test_end_rule_on_differences_matches_linear_continuation():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "edge_rule.cu")
        exe = os.path.join(tmp, "edge_rule")
        with open(src, "w") as f:
            f.write(PROGRAM)
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
                               "-I", CSRC, src, "-o", exe])
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
