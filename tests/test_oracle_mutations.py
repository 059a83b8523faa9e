"""Planted mistakes in the oracle must fail its pins (CPU only).

Each case copies oracle/hsg_oracle.c, plants one plausible mistake (a dropped
term, a wrong sign, a wrong bond index, a swapped operand, a wrong constant
or order), builds the copy, and runs tests/test_oracle_pins.py against it in
a subprocess (HSG_ORACLE_LIB points the oracle package at the copy).  The
golden-fixture pin is left out: it holds the oracle's own output, so it
would catch every change and prove nothing about the other pins.  A control
case builds the unchanged source the same way and must pass.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hsg_oracle.c")

_MAIN = ("    if (sch->kind == ORACLE_MET || sch->kind == ORACLE_HB || sch->kind == ORACLE_MET_OR) {\n"
         "      oracle_half_sweep(L, J, s, sch->kind, 0, &p, NULL);\n"
         "      oracle_half_sweep(L, J, s, sch->kind, 1, &p, NULL);\n"
         "    }\n")
_OR = ("    for (int o = 0; o < sch->n_or; ++o) {\n"
       "      oracle_half_sweep(L, J, s, ORACLE_OR, 0, &p, NULL);\n"
       "      oracle_half_sweep(L, J, s, ORACLE_OR, 1, &p, NULL);\n"
       "    }\n")

# (what is planted, text in the source, replacement)
MUTATIONS = [
    ("local field: the -d term dropped",
     "h[a] += j_up * s[3 * up + a] + j_dn * s[3 * dn + a];", "h[a] += j_up * s[3 * up + a];"),
    ("local field: the -d bond read at the site itself", "double j_dn = J[3 * dn + d];", "double j_dn = J[3 * i + d];"),
    ("energy: sign", "e -= J[3 * i + d] * dot;", "e += J[3 * i + d] * dot;"),
    ("energy: the z bonds dropped",
     "for (int d = 0; d < 3; ++d) {\n      int64_t up = neighbour(L, i, d, +1);\n      double dot",
     "for (int d = 0; d < 2; ++d) {\n      int64_t up = neighbour(L, i, d, +1);\n      double dot"),
    ("over-relaxation: factor 2 dropped", "double f = 2.0 * dot3(s, h) / hh;", "double f = dot3(s, h) / hh;"),
    ("Metropolis: sign of dE", "de -= (prop[a] - cur[a]) * h[a];", "de += (prop[a] - cur[a]) * h[a];"),
    ("Metropolis: ball radius u2 instead of cbrt(u2)", "double rho = cbrt(u2);", "double rho = u2;"),
    ("Metropolis: acceptance inverted", "if (u3 < pacc) {", "if (u3 > pacc) {"),
    ("heat-bath: expm1(-x) instead of expm1(-2x)", "expm1(-2.0 * x)) / x;", "expm1(-x)) / x;"),
    ("heat-bath: azimuth from u0",
     "double st = sqrt(fmax(sv * (2.0 - sv), 0.0));\n  double phi = 2.0 * ORACLE_PI * u1;",
     "double st = sqrt(fmax(sv * (2.0 - sv), 0.0));\n  double phi = 2.0 * ORACLE_PI * u0;"),
    ("heat-bath: sign of a frame component", "e2[2] = -n[1];", "e2[2] = n[1];"),
    ("checkerboard: colours swapped", "return (x + y + z) % 2;", "return (x + y + z + 1) % 2;"),
    ("sweep: over-relaxation before the main update", _MAIN + _OR, _OR + _MAIN),
    ("Philox: a Weyl constant", "weyl1 = 0xBB67AE85u;", "weyl1 = 0xBB67AE87u;"),
    ("uniform: 24 bits instead of 23", "uint32_t m = r >> 9;", "uint32_t m = r >> 8;"),
    ("sphere point: z = u0", "double z = 2.0 * u0 - 1.0;", "double z = u0;"),
    ("renormalisation by |s|^2", "double nrm = sqrt(dot3(&s[3 * i], &s[3 * i]));",
     "double nrm = dot3(&s[3 * i], &s[3 * i]);"),
    ("Box-Muller: J_z from u1", "out[2] = b * cos(2.0 * ORACLE_PI * u3);", "out[2] = b * cos(2.0 * ORACLE_PI * u1);"),
    ("key: sample and replica transposed", "(2u * sample + replica)", "(2u * replica + sample)"),
    ("counter: colour and hit fields swapped", "((uint32_t)colour << 16) | (uint32_t)hit;",
     "((uint32_t)hit << 16) | (uint32_t)colour;"),
    ("fused pass: the old spin reflected", "update_or(mid, h, out);", "update_or(s, h, out);"),
    ("heat-bath: cos(theta) = s - 1", "double ct = 1.0 - sv;", "double ct = sv - 1.0;"),
]


def run_pins(tmp_path, source: str) -> subprocess.CompletedProcess:
    c = tmp_path / "hsg_oracle_copy.c"
    c.write_text(source)
    so = tmp_path / "libhsg_oracle_copy.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"],
                   check=True)
    env = dict(os.environ, HSG_ORACLE_LIB=str(so))
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", "test_oracle_pins.py"), "-x", "-q",
                           "-k", "not golden", "-p", "no:cacheprovider"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def test_control_copy_passes_the_pins(tmp_path):
    r = run_pins(tmp_path, open(SRC).read())
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, what, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique or missing: {what}"
    r = run_pins(tmp_path, src.replace(old, new))
    assert r.returncode == 1, f"{what}: no pin failed\n{r.stdout[-3000:]}"
