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
    ("tile rectangle at the tile edge", BLEND, "*x0 = tile * tx + 0.5;", "*x0 = tile * tx;"),
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
    ('distance without its z term', CUT, 'float d2 = (dx * dx + dy * dy) + dz * dz;\n    float lhs',
     'float d2 = (dx * dx + dy * dy);\n    float lhs'),
    ('Jacobian clamp at 1.0', PROJ, 'double limx = 1.3 * (0.5',
     'double limx = 1.0 * (0.5'),
    ('Jacobian not clamped', PROJ, 'double tx = fmin(limx, fmax(-limx, p[0] / z));',
     'double tx = p[0] / z;'),
    ('conic a and c swapped', PROJ, 'P->conic[0] = s11 / det;',
     'P->conic[0] = s00 / det;'),
    ('covariance rotated by R twice', PROJ, 'acc += RS[3 * r + k] * R[3 * c + k];',
     'acc += RS[3 * r + k] * R[3 * k + c];'),
    ('no principal point', PROJ, 'P->u = fx * p[0] / z + cam->cx;',
     'P->u = fx * p[0] / z;'),
    ('colour without +0.5', PROJ, '        acc += 0.5;\n',
     ''),
    ('colour not clamped at 0', PROJ, 'P->rgb[ch] = acc > 0.0 ? acc : 0.0;',
     'P->rgb[ch] = acc;'),
    ('SH sin for m > 0', PROJ, 'else if (m > 0) v = sqrt(2.0) * K * P * cos(m * phi);',
     'else if (m > 0) v = sqrt(2.0) * K * P * sin(m * phi);'),
    ('SH without sqrt 2', PROJ, 'else v = sqrt(2.0) * K * P * sin(am * phi);',
     'else v = K * P * sin(am * phi);'),
    ('no Condon-Shortley phase', PROJ, 'pmm *= -(2.0 * i - 1.0) * sx;',
     'pmm *= (2.0 * i - 1.0) * sx;'),
    ('depth key from a column of R', PROJ, 'float zk = (cam->R[6] * dxf + cam->R[7] * dyf) + cam->R[8] * dzf;',
     'float zk = (cam->R[2] * dxf + cam->R[5] * dyf) + cam->R[8] * dzf;'),
    ('threshold sign', BLEND, 'P->thr = log(ORC_ALPHA_MIN) - log(',
     'P->thr = -log(ORC_ALPHA_MIN) + log('),
    ('rho cross-term sign', BLEND, 'return -0.5 * (conic[0] * dx * dx + conic[2] * dy * dy) - conic[1] * dx * dy;',
     'return -0.5 * (conic[0] * dx * dx + conic[2] * dy * dy) + conic[1] * dx * dy;'),
    ('rho without 1/2', BLEND, 'return -0.5 * (conic[0]',
     'return -1.0 * (conic[0]'),
    ('tile rectangle not clipped to the image', BLEND, '*x1 = fmin(tile * tx + tile - 0.5, (double)cam->width - 0.5);',
     '*x1 = tile * tx + tile - 0.5;'),
    ('rho_max without the inside case', BLEND, 'if (u >= x0 && u <= x1 && v >= y0 && v <= y1) return 0.0;',
     ''),
    ('box radius without the factor 2', BLEND, 'double r2 = 2.0 * (log(P->theta)',
     'double r2 = 1.0 * (log(P->theta)'),
    ('box x extent from the y variance', BLEND, 'double bx = sqrt(r2 * P->cov[0])',
     'double bx = sqrt(r2 * P->cov[2])'),
    ('order without depth', BLEND, 'if (x->zkey != y->zkey) return x->zkey < y->zkey ? -1 : 1;',
     ''),
    ('back to front', BLEND, 'if (x->zkey != y->zkey) return x->zkey < y->zkey ? -1 : 1;',
     'if (x->zkey != y->zkey) return x->zkey > y->zkey ? -1 : 1;'),
    ('no alpha* skip', BLEND, '            if (alpha < ORC_ALPHA_MIN) continue;\n',
     ''),
    ('termination after adding', BLEND, '        if (Tn < ORC_T_MIN) break;\n        for (int ch = 0; ch < 3; ++ch) C[ch] += alpha * T * g->rgb[ch];',
     '        for (int ch = 0; ch < 3; ++ch) C[ch] += alpha * T * g->rgb[ch];\n        if (Tn < ORC_T_MIN) break;'),
    ('pixel corner, not centre', BLEND, 'orc_blend_pixel(F->proj, list, n, x + 0.5, y + 0.5,',
     'orc_blend_pixel(F->proj, list, n, x, y,'),
    ('frustum normals from R, not R^T', FRUSTUM, 'double acc = (double)cam->R[0 * 3 + j] * a[i][0];\n            acc = fma((double)cam->R[1 * 3 + j], a[i][1], acc);\n            acc = fma((double)cam->R[2 * 3 + j], a[i][2], acc);',
     'double acc = (double)cam->R[j * 3 + 0] * a[i][0];\n            acc = fma((double)cam->R[j * 3 + 1], a[i][1], acc);\n            acc = fma((double)cam->R[j * 3 + 2], a[i][2], acc);'),
    ('right plane facing out', FRUSTUM, '{-(double)cam->fx, 0.0, (W - cam->cx) + g}',
     '{(double)cam->fx, 0.0, (W - cam->cx) + g}'),
    ('plane offset sign', FRUSTUM, 'planes[4 * i + 3] = (float)(o + oc[i]);',
     'planes[4 * i + 3] = (float)(-o + oc[i]);'),
    ('no near plane', FRUSTUM, 'double oc[5] = {cam->z_near, 0.0, 0.0, 0.0, 0.0};',
     'double oc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};'),
    ('bottom plane from cy, not H - cy', FRUSTUM, '{0.0, -(double)cam->fy, (H - cam->cy) + g}',
     '{0.0, -(double)cam->fy, (double)cam->cy + g}'),
    ('only the near plane tested', FRUSTUM, 'if (!(sd >= 0.0f)) return 0;',
     'if (!(sd >= 0.0f) && i == 0) return 0;'),
    ('size ratio without the square root', INTERP, 'return sqrtf(q);',
     'return q;'),
    ('node and parent swapped', INTERP, 'float an = orc_size_ratio(s, n, cam), ap = orc_size_ratio(s, p, cam);',
     'float ap = orc_size_ratio(s, n, cam), an = orc_size_ratio(s, p, cam);'),
    ('mean moved away from the parent', INTERP, 'mf[j] = mf[j] + wd;',
     'mf[j] = mf[j] - wd;'),
    ('SH not interpolated', INTERP, 'for (int j = 0; j < 3 * K; ++j) shn[j] += wd * ((double)s->sh[(size_t)p * K * 3 + j] - shn[j]);',
     ''),
    ('covariance not interpolated', INTERP, 'for (int j = 0; j < 6; ++j) c6[j] += wd * ((double)s->cov6[6 * (size_t)p + j] - c6[j]);',
     ''),
    ('table index rounded up', LUT, 'float q = nearbyintf((float)rho * lut_scale);',
     'float q = ceilf((float)rho * lut_scale);'),
    ('table scaled by ln 255, not 5.55', LUT, '-(float)lut_m / 5.55f',
     '-(float)lut_m / 5.541f'),
    ('table of m + 1 intervals', LUT, 'exp(-5.55 * (double)i / (double)lut_m)',
     'exp(-5.55 * (double)i / (double)(lut_m + 1))'),
    ('table with a second alpha* test', LUT, '            alpha = fmin(ORC_ALPHA_MAX, g->theta * exp(-5.55 * (double)i / (double)lut_m));\n',
     '            alpha = fmin(ORC_ALPHA_MAX, g->theta * exp(-5.55 * (double)i / (double)lut_m));\n            if (alpha < ORC_ALPHA_MIN) continue;\n'),
    ('table without the alpha cap', LUT, 'alpha = fmin(ORC_ALPHA_MAX, g->theta * exp(-5.55 * (double)i / (double)lut_m));',
     'alpha = g->theta * exp(-5.55 * (double)i / (double)lut_m);'),
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
