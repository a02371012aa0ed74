"""Mutation check of the oracle's pins (test infrastructure).

Plants one plausible mistake at a time in a copy of hj_oracle.c (a flipped
sign, a swapped weight, a dropped term or option), compiles the copy into a
temporary directory, and runs the CPU pins against it through
HJ_ORACLE_LIB.  The oracle's Python parts (translation, safety filter) get
the same treatment through a modified copy of the package placed first on
the import path.  Every mistake must fail at least one pin.  The committed
sources are never modified.

    python oracle/mutation_check.py
"""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PINS = ["tests/test_oracle_pins.py", "tests/test_golden.py", "tests/test_oracle_properties.py"]

# (mistake, [(text in hj_oracle.c, replacement), ...])
MUTATIONS = [
    ("Lax-Friedrichs dissipation with the wrong sign",
     [("L += alpha[d] * 0.5 * (pp[d] - pm[d]);", "L -= alpha[d] * 0.5 * (pp[d] - pm[d]);")]),
    ("TVD-RK3 stage 2 weights 1/2, 1/2", [("0.75 * W[i] + 0.25 *", "0.5 * W[i] + 0.5 *")]),
    ("TVD-RK3 stage 3 weights swapped",
     [("W[i] / 3.0 + 2.0 / 3.0 *", "2.0 * W[i] / 3.0 + 1.0 / 3.0 *")]),
    ("no clamp against l", [("double wn = fmin(w3, l[i]);", "double wn = w3;")]),
    ("WENO5 linear weights swapped",
     [("double a1 = 0.1 /", "double a1 = 0.3 /"), ("double a3 = 0.3 /", "double a3 = 0.1 /")]),
    ("WENO5 smoothness indicator without 13/12",
     [("double s1 = 13.0 / 12.0 *", "double s1 = 1.0 *")]),
    ("ENO2 takes the larger second difference",
     [("(fabs(a) <= fabs(b)) ? a : b;", "(fabs(a) >= fabs(b)) ? a : b;")]),
    ("ENO2 correction without the 1/2",
     [("*pm = (v[2] - v[1]) / h + m1 / (2.0 * h);", "*pm = (v[2] - v[1]) / h + m1 / h;")]),
    ("constant instead of linear ghosts", [("return w0 + (double)(-j) * (w0 - w1);", "return w0;")]),
    ("the disturbance maximises",
     [("if (s < worst) worst = s;", "if (s > worst || worst == INFINITY) worst = s;")]),
    ("the control minimises",
     [("if (worst > best) best = worst;", "if (worst < best || best == -INFINITY) best = worst;")]),
    ("alpha from one node only",
     [("  for (int i = 0; i < P->ndim; ++i) alpha[i] = 0.0;\n  for (long pt = 0; pt < npts; ++pt) {",
       "  for (int i = 0; i < P->ndim; ++i) alpha[i] = 0.0;\n  for (long pt = 0; pt < 1; ++pt) {")]),
    ("CFL doubled", [("return (s > 0.0) ? cfl / s : 0.0;", "return (s > 0.0) ? 2.0 * cfl / s : 0.0;")]),
    ("interpolation weights swapped",
     [("wgt *= bit ? fr[d] : 1.0 - fr[d];", "wgt *= bit ? 1.0 - fr[d] : fr[d];")]),
    ("node gradient over h instead of 2h",
     [("else g[pt] = (W[pt + s] - W[pt - s]) / (2.0 * h);",
       "else g[pt] = (W[pt + s] - W[pt - s]) / h;")]),
    ("box margin inside takes the farther face",
     [("double in_d = fmin(x[d] - lo, hi - x[d]);", "double in_d = fmax(x[d] - lo, hi - x[d]);")]),
    ("band of the stop test ignored",
     [("if (o->band > 0.0 && fmin(fabs(W[i]), fabs(snap[i])) > o->band) continue;", "")]),
    ("monotone clamp ignored", [("if (clamp == OR_CLAMP_MONOTONE) wn = fmin(wn, W[i]);", "")]),
    ("warm start ignores the prior",
     [("W[i] = o->warm ? fmin(W[i], l[i]) : l[i];", "W[i] = l[i];")]),
    ("state-dependent disturbance bound ignored",
     [("lo[j] = P->dflo ? P->dflo[j * npts + pt] : P->d_lo[j];", "lo[j] = P->d_lo[j];"),
      ("hi[j] = P->dfhi ? P->dfhi[j * npts + pt] : P->d_hi[j];", "hi[j] = P->d_hi[j];")]),
    ("x/y control enters with the wrong sign",
     [("f[3] = -q[2] * x[2] + q[3] * u[0];", "f[3] = -q[2] * x[2] - q[3] * u[0];")]),
    ("x/y angle damping with the wrong sign",
     [("f[2] = -q[1] * x[2] + x[3];", "f[2] = q[1] * x[2] + x[3];")]),
]


# the same for binding.py
PY_MUTATIONS = [
    ("translation reads the source at x + s",
     [("Y = X - np.asarray(shift, dtype=np.float64)[None, :]",
       "Y = X + np.asarray(shift, dtype=np.float64)[None, :]")]),
    ("translated prior not clamped by l",
     [("out[inside] = np.minimum(query_value(src, Ws, Y[inside]), l[inside])",
       "out[inside] = query_value(src, Ws, Y[inside])")]),
    ("z control gain on the wrong axis", [("b[1] = spec.params[0]", "b[0] = spec.params[0]")]),
    ("x control gain on the wrong axis", [("b[3] = spec.params[3]", "b[2] = spec.params[3]")]),
    ("decomposed value is the maximum", [("w = np.minimum(w, wk)", "w = np.maximum(w, wk)")]),
    ("filter switches above the level", [("on = wk <= level", "on = wk >= level")]),
    ("bang-bang bounds swapped",
     [("us = np.where(s > 0, uhi, np.where(s < 0, ulo,", "us = np.where(s > 0, ulo, np.where(s < 0, uhi,")]),
]


def _run_pins(env, cwd) -> str:
    """Runs the pins; returns the first failing test, or '' when all pass.
    cwd is a scratch directory: `python -m pytest` puts its working
    directory first on sys.path, which must not hold the real oracle when a
    modified copy is to be imported."""
    r = subprocess.run([sys.executable, "-m", "pytest", *[os.path.join(ROOT, p) for p in PINS],
                        "-q", "-x", "-m", "not gpu", "-p", "no:cacheprovider"], cwd=cwd, env=env,
                       capture_output=True, text=True)
    if r.returncode == 0:
        return ""
    failed = [l.split("::", 1)[1] for l in r.stdout.splitlines() if l.startswith("FAILED")]
    return failed[0].split(" ")[0] if failed else "(error)"


def main() -> int:
    src = open(os.path.join(HERE, "hj_oracle.c")).read()
    survived = 0
    with tempfile.TemporaryDirectory() as tmp:
        # a built copy of the unmodified library for the Python mutations
        base_so = os.path.join(tmp, "base.so")
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", base_so, os.path.join(HERE, "hj_oracle.c"), "-lm"])
        for k, (name, edits) in enumerate(MUTATIONS):
            text = src
            for a, b in edits:
                if a not in text:
                    raise SystemExit("mutation %r: pattern not found" % name)
                text = text.replace(a, b, 1)
            c = os.path.join(tmp, "m%d.c" % k)
            so = os.path.join(tmp, "m%d.so" % k)
            open(c, "w").write(text)
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                                   "-o", so, c, "-lm"])
            first = _run_pins(dict(os.environ, HJ_ORACLE_LIB=so), tmp)
            if not first:
                survived += 1
                print("SURVIVED  %s" % name)
            else:
                print("caught    %-48s by %s" % (name, first))
        binding = open(os.path.join(HERE, "binding.py")).read()
        for k, (name, edits) in enumerate(PY_MUTATIONS):
            text = binding
            for a, b in edits:
                if a not in text:
                    raise SystemExit("mutation %r: pattern not found" % name)
                text = text.replace(a, b, 1)
            pkg = os.path.join(tmp, "py%d" % k, "oracle")
            os.makedirs(pkg)
            open(os.path.join(pkg, "binding.py"), "w").write(text)
            open(os.path.join(pkg, "__init__.py"), "w").write(
                open(os.path.join(HERE, "__init__.py")).read())
            path = os.pathsep.join([os.path.dirname(pkg), ROOT, os.environ.get("PYTHONPATH", "")])
            first = _run_pins(dict(os.environ, HJ_ORACLE_LIB=base_so, PYTHONPATH=path), tmp)
            if not first:
                survived += 1
                print("SURVIVED  %s" % name)
            else:
                print("caught    %-48s by %s" % (name, first))
    total = len(MUTATIONS) + len(PY_MUTATIONS)
    print("%d of %d mistakes caught" % (total - survived, total))
    return 1 if survived else 0


if __name__ == "__main__":
    sys.exit(main())
