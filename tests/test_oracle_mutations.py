"""Planted mistakes in the oracle must fail its pins.

Each case copies oracle/pic_oracle.cpp, plants one plausible mistake (a dropped
or doubled term, a wrong sign, a swapped index or weight, a missing mass), builds
the copy on the CPU and runs tests/test_oracle_pins.py and
tests/test_oracle_pins_tsc.py against it in a subprocess.  The pins are only worth something if every such copy fails them.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pic_oracle.cpp")

MUTATIONS = [
    ("VB correction term", "sigma * d[p] * d[r] / T(12.0)", "sigma * d[p] * d[r] / T(6.0)"),
    ("VB correction sign", "double sigma = (s1 == s2) ? 1.0 : -1.0;", "double sigma = (s1 == s2) ? -1.0 : 1.0;"),
    ("VB transverse weight", "T wp = s1 ? m[p] : T(1.0) - m[p];", "T wp = s1 ? T(1.0) - m[p] : m[p];"),
    ("VB crossing face", "double face = std::max(c0, c1);", "double face = std::min(c0, c1);"),
    ("Boris cross product", "up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);",
     "up[1] = um[1] + (um[0] * t[2] - um[2] * t[0]);"),
    ("Boris s factor", "s[a] = T(2.0) * t[a] / (T(1.0) + t2);", "s[a] = T(2.0) * t[a] / (T(1.0) + t2 * t2);"),
    ("Boris mass", "double h = 0.5 * q * dt / m;", "double h = 0.5 * q * dt;"),
    ("B staggering", "inline double stagB(int comp, int axis) { return comp == axis ? 0.0 : 0.5; }",
     "inline double stagB(int comp, int axis) { return comp == axis ? 0.5 : 0.0; }"),
    ("curl cell size", "(at(g, E[2], i + 1, j, k) - at(g, E[2], i, j, k)) * rx;",
     "(at(g, E[2], i + 1, j, k) - at(g, E[2], i, j, k)) * ry;"),
    ("Ampere current sign", "nE[1][o] = E[1][o] + dt * (cy - J[1][o]);", "nE[1][o] = E[1][o] + dt * (cy + J[1][o]);"),
    ("gather weight", "T wx = bx ? f[0] : T(1.0) - f[0];", "T wx = bx ? T(1.0) - f[0] : f[0];"),
    ("move uses u not v", "T disp = g.dt * u[a] / gam;", "T disp = g.dt * u[a];"),
    ("segment midpoint", "for (int e = 0; e < 3; ++e) m[e] = a[e] + T(0.5) * d[e];",
     "for (int e = 0; e < 3; ++e) m[e] = a[e] + d[e];"),
    ("kinetic energy rest mass", "s += sp.w[p] * (gam - T(1.0));", "s += sp.w[p] * gam;"),
    # second-order form factor and Esirkepov current
    ("TSC centre weight", "w[1] = T(0.75) - delta * delta;", "w[1] = T(0.75) + delta * delta;"),
    ("TSC nearest node", "double fl = std::floor(val(s) + 0.5);", "double fl = std::floor(val(s));"),
    ("Esirkepov cross term", "dS[p][jp] * dS[r][jr] / T(3.0);", "dS[p][jp] * dS[r][jr] / T(2.0);"),
    ("Esirkepov half term", "T(0.5) * dS[p][jp] * S0[r][jr]", "dS[p][jp] * S0[r][jr]"),
    ("Esirkepov current sign", "T(-1.0) * qfac[c] * running", "qfac[c] * running"),
    ("Esirkepov running sum", "running += dS[c][i] * transverse;", "running = dS[c][i] * transverse;"),
    ("Esirkepov factored centre change", "dS[a][2] = T(-1.0) * d[a] * (delta0 + delta1);",
     "dS[a][2] = T(-1.0) * d[a] * (delta0 - delta1);"),
    ("TSC rho weight", "sp->q * sp->w[p] / dV * (w[0][a] * w[1][b] * w[2][c])",
     "sp->q * sp->w[p] / dV * (w[0][a] * w[1][b] * w[2][b])"),
    ("damping staggering", "double off = isB ? stagB(c, a) : stagE(c, a);",
     "double off = isB ? stagE(c, a) : stagB(c, a);"),
    ("damping distance", "double dist = std::min(p, (double)n - p);", "double dist = std::min(p, (double)n - 1 - p);"),
]


@pytest.mark.parametrize("label,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_pins(label, old, new, tmp_path):
    src = open(SRC).read()
    assert old in src, "mutation anchor not found: %s" % label
    mut = tmp_path / "mut.cpp"
    mut.write_text(src.replace(old, new, 1))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                           str(lib), str(mut)])
    env = dict(os.environ, PIC_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_pins_tsc.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "planted mistake '%s' passed every pin:\n%s" % (label, r.stdout[-2000:])
