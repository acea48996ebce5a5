"""The oracle's pins catch plausible mistakes.  Each case compiles a copy of
oracle.c with one mistake planted (in a temporary directory: the source in
the tree is never touched), loads it through ORACLE_LIB in a child pytest
run of the pin file that covers that step, and requires that run to fail.
A control build of the unmodified source must pass the same files."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

CUT, PROJ, BLEND = "tests/test_oracle_cut.py", "tests/test_oracle_projection.py", "tests/test_oracle_blend.py"
FRUSTUM, INTERP, LUT = "tests/test_oracle_frustum.py", "tests/test_oracle_interp.py", "tests/test_oracle_lut.py"

# (name, pin file, original text, planted mistake)
MUTANTS = [
    ("granularity k = t, not t^2", CUT, "    return t * t;\n}", "    return t;\n}"),
    ("granularity boundary <=", CUT, "if (!(lhs < s->radius2[n])) return 0;", "if (!(lhs <= s->radius2[n])) return 0;"),
    ("Jacobian sign", PROJ, "-fx * tx / z, 0.0", "fx * tx / z, 0.0"),
    ("conic off-diagonal sign", PROJ, "P->conic[1] = -s01 / det;", "P->conic[1] = s01 / det;"),
    ("no dilation", PROJ, "double s00 = C2[0] + ORC_DILATE, s01 = 0.5 * (C2[1] + C2[2]), s11 = C2[3] + ORC_DILATE;",
     "double s00 = C2[0], s01 = 0.5 * (C2[1] + C2[2]), s11 = C2[3];"),
    ("SH view direction reversed", PROJ, "double dir[3] = {d[0] / nd, d[1] / nd, d[2] / nd};",
     "double dir[3] = {-d[0] / nd, -d[1] / nd, -d[2] / nd};"),
    ("near plane inclusive", PROJ, "if (!(zk > cam->z_near)) return;", "if (!(zk >= cam->z_near)) return;"),
    ("tile rectangle at the tile edge", BLEND, "*x0 = ORC_TILE * tx + 0.5;", "*x0 = ORC_TILE * tx;"),
    ("no Gaussian-level filter", BLEND, "if (P->theta < ORC_ALPHA_MIN) return; /* Gaussian-level filter */", ""),
    ("rho_max edge not clamped", BLEND, "double dy = orc_clamp(-b * dx / c, y0 - v, y1 - v);", "double dy = y0 - v;"),
    ("equal depths by descending id", BLEND, "if (x->node != y->node) return x->node < y->node ? -1 : 1;",
     "if (x->node != y->node) return x->node > y->node ? -1 : 1;"),
    ("no alpha cap", BLEND, "alpha = fmin(ORC_ALPHA_MAX, g->theta * exp(rho));", "alpha = g->theta * exp(rho);"),
    ("no early termination", BLEND, "        if (Tn < ORC_T_MIN) break;\n", ""),
    ("colour weighted by T'", BLEND, "C[ch] += alpha * T * g->rgb[ch];", "C[ch] += alpha * Tn * g->rgb[ch];"),
    ("frustum box corner swapped", FRUSTUM, "float X = p[0] >= 0.0f ? box[3] : box[0];",
     "float X = p[0] >= 0.0f ? box[0] : box[3];"),
    ("frustum guard dropped", FRUSTUM, "(double)cam->cx + g}", "(double)cam->cx}"),
    ("interpolation weight 1 - w", INTERP, "return fminf(1.0f, fmaxf(0.0f, w));",
     "return fminf(1.0f, fmaxf(0.0f, 1.0f - w));"),
    ("interpolated opacity = parent's", INTERP,
     "double share = -expm1(log1p(-(double)s->opacity[p]) / (double)s->n_child[p]);",
     "double share = s->opacity[p];"),
    ("table index floored", LUT, "float q = nearbyintf((float)rho * lut_scale);",
     "float q = floorf((float)rho * lut_scale);"),
    ("table without Eq. 4 first", LUT, "            if (rho < g->thr) continue; /* Eq. 4 */\n", ""),
]


def _build(tmp_path, text, tag):
    c = tmp_path / ("oracle_%s.c" % tag)
    c.write_text(text)
    so = tmp_path / ("liboracle_%s.so" % tag)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(c), "-lm"])
    return str(so)


def _pins(lib, files):
    env = dict(os.environ, ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", *files, "-x", "-q", "-p", "no:cacheprovider"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_control_build_passes_the_pins(tmp_path):
    r = _pins(_build(tmp_path, open(SRC).read(), "control"), sorted({m[1] for m in MUTANTS}))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,pin,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, pin, orig, bad):
    src = open(SRC).read()
    assert src.count(orig) == 1, "the planted text no longer matches oracle.c: " + name
    r = _pins(_build(tmp_path, src.replace(orig, bad), "mutant"), [pin])
    assert r.returncode == 1, (name, r.stdout[-1500:])  # 1: pins failed (not a crash or a usage error)
