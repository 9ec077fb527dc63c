"""The oracle's pins are strong enough: each plausible slip planted in a copy
of the C oracle (a dropped term, a flipped sign, a wrong index, a min for a
max) makes at least one pin in test_oracle_pins.py fail.

Mistakes are planted only in a temporary copy of the oracle, compiled on the
CPU; the real oracle library is not touched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fv_oracle.c")

# (what the slip is, original text, planted text)
MUTATIONS = [
    ("energy flux printed without the velocity (Eq. 2 as typeset)",
     "f[d + 1] = (q[d + 1] + p) * u;", "f[d + 1] = (q[d + 1] + p) / rho;"),
    ("dissipation sign flipped (Eq. 4)",
     "F[v] = 0.5 * ((fL[v] + fR[v]) - a * (qR[v] - qL[v]));",
     "F[v] = 0.5 * ((fL[v] + fR[v]) + a * (qR[v] - qL[v]));"),
    ("min instead of max wave speed (Eq. 5)",
     "double a = lamL > lamR ? lamL : lamR;\n  for", "double a = lamL < lamR ? lamL : lamR;\n  for"),
    ("update sign flipped (Eq. 3)", "qo[v] = qc[v] - r * acc[v];", "qo[v] = qc[v] + r * acc[v];"),
    ("kinetic energy factor 1/2 dropped", "(q[d + 1] - 0.5 * jj / rho)", "(q[d + 1] - jj / rho)"),
    ("transverse faces dropped", "acc[v] = acc[v] + (Fp[v] - Fm[v]);",
     "acc[v] = acc[v] + (Fp[v] - Fm[v]) * (k == 0);"),
    ("pressure on every momentum component", "f[1 + k] = q[1 + k] * u + (k == dir ? p : 0.0);",
     "f[1 + k] = q[1 + k] * u + p;"),
    ("gamma dropped from the sound speed", "double c = sqrt(gamma * p / rho);",
     "double c = sqrt(p / rho);"),
    ("right neighbour index off by one", "cp[k] += 1;", "cp[k] += 0;"),
    ("halo source layer off by one", "src = side == 0 ? dst + p : dst - p;",
     "src = side == 0 ? dst + p : dst - p + 1;"),
    ("wall forgets to negate the normal momentum",
     "if (nb == -2 && 1 + k < s) qd[1 + k] = -qs[1 + k];", ""),
    ("eigenvalue faces miss the low halo layer", "c[k2] = (k2 == k ? h - 1 : h) + rem % len;",
     "c[k2] = h + rem % len;"),
    ("conservation sums over the whole box, halo included",
     "for (int k = 0; k < d; ++k) ncell *= p;\n    for (int t = 0; t < ncell; ++t) {\n"
     "      int c[3] = {0, 0, 0};\n      int rem = t;\n      for (int k = 0; k < d; ++k) {\n"
     "        c[k] = h + rem % p;\n        rem /= p;",
     "for (int k = 0; k < d; ++k) ncell *= ne;\n    for (int t = 0; t < ncell; ++t) {\n"
     "      int c[3] = {0, 0, 0};\n      int rem = t;\n      for (int k = 0; k < d; ++k) {\n"
     "        c[k] = rem % ne;\n        rem /= ne;"),
    ("conservation sums read the interior at the wrong row stride",
     "const double *qc = Q + cell_index(c, d, ne) * s;\n"
     "      for (int v = 0; v < s; ++v) acc[v] = acc[v] + qc[v];",
     "const double *qc = Q + cell_index(c, d, p) * s;\n"
     "      for (int v = 0; v < s; ++v) acc[v] = acc[v] + qc[v];"),
]


@pytest.mark.parametrize("name,orig,planted", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, orig, planted):
    src = open(SRC).read()
    assert orig in src, "mutation anchor no longer in the oracle"
    csrc = tmp_path / "mut.c"
    csrc.write_text(src.replace(orig, planted, 1))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared", "-o",
                    str(so), str(csrc), "-lm"], check=True)
    env = dict(os.environ, FV_ORACLE_SO_OVERRIDE=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake not caught: {name}\n{r.stdout[-2000:]}"
