"""Planted mistakes: each mutant is a copy of the oracle source with one plausible
error (a dropped term, a wrong sign, a transposed index, a wrong weight or bound).
The pins must reject every mutant.  The mutants are compiled on the CPU into a
temporary directory; the oracle in the repository is not touched.  CPU only.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rgeo_oracle.c")

MUTANTS = {
    "eq53_sign": ("Gam[mm * 9 + i * 3 + j] = gr[mm] * H[3 * i + j] / den;",
                  "Gam[mm * 9 + i * 3 + j] = -gr[mm] * H[3 * i + j] / den;", "christoffel"),
    "hessian_dropped_term": ("hess[3 * i + j] += fk * (d[i] * d[j] / (s2[i] * s2[j]) - dij);",
                             "hess[3 * i + j] += fk * (d[i] * d[j] / (s2[i] * s2[j]));", "finite_diff"),
    "minors_transposed": ("Jinv[3 * m + s] = sign * dm / dJ;", "Jinv[3 * s + m] = sign * dm / dJ;",
                          "minors or twist"),
    "rk4_weight": ("x[i] = x[i] + h / 6.0 * (v1[i] + 2.0 * v2[i] + 2.0 * v3[i] + v4[i]);",
                   "x[i] = x[i] + h / 6.0 * (v1[i] + 2.0 * v2[i] + 1.0 * v3[i] + v4[i]);", "straight"),
    "rk4_stage": ("x4[i] = x[i] + h * v3[i]; v4[i] = v[i] + h * a3[i];",
                  "x4[i] = x[i] + h * v2[i]; v4[i] = v[i] + h * a3[i];", "convergence or twist_geodesics"),
    "twist_hessian_sign": ("H[1 * 9 + 1 * 3 + 2] = H[1 * 9 + 2 * 3 + 1] = -k * s;",
                           "H[1 * 9 + 1 * 3 + 2] = H[1 * 9 + 2 * 3 + 1] = k * s;", "twist"),
    "sphere_smax_inclusive": ("  if (!(s < smax)) return 0;\n  *s_out = s;\n  return 1;\n}\n\n/* Segment against",
                              "  if (!(s <= smax)) return 0;\n  *s_out = s;\n  return 1;\n}\n\n/* Segment against",
                              "sphere"),
    "skip_to_exit": ("double t = (-B - sqrt(disc)) / A;", "double t = (-B + sqrt(disc)) / A;", "skip"),
    "camera_flipped": ("double py = (1.0 - 2.0 * (j + 0.5) / H) * th;",
                       "double py = (2.0 * (j + 0.5) / H - 1.0) * th;", "camera"),
    "no_g_unit": ("double v[3] = {d[0] / nd, d[1] / nd, d[2] / nd};",
                  "double v[3] = {d[0], d[1], d[2]};", "g_unit"),
    "watertight_edge_sign": ("double V = Ax * Cy - Ay * Cx;", "double V = Ay * Cx - Ax * Cy;",
                             "triangle or watertight or bvh"),
    "eq63_dropped_term": ("          for (int r = 0; r < 3; r++) acc += Jj[3 * s + r] * H[9 * r + 3 * a + b];\n", "",
                          "local"),
    "eq63_transposed_jacobian": ("acc += J[3 * k + a] * Hj[9 * s + 3 * k + l] * J[3 * l + b];",
                                 "acc += J[3 * a + k] * Hj[9 * s + 3 * k + l] * J[3 * b + l];", "local"),
    "jinv_product_order": ("t += inv[3 * r + k] * Jinv[3 * k + c];", "t += Jinv[3 * r + k] * inv[3 * k + c];",
                           "local"),
    "fog_skip_arc": ("      for (int c = 0; c < 3; c++) x[c] = x[c] + t * v[c];\n      arc += t;\n",
                     "      for (int c = 0; c < 3; c++) x[c] = x[c] + t * v[c];\n", "fog"),
    "fog_step_arc": ("    arc += jb->h;\n  }", "  }", "fog"),
    "local_field_term": ("hs[3 * i + j] * V[s] + gr[j] * B[3 * s + i] + gr[i] * B[3 * s + j];",
                         "hs[3 * i + j] * V[s] + gr[j] * B[3 * s + i];", "local"),
    # full traces
    "hit_at_segment_end": ("      for (int c = 0; c < 3; c++) { P[c] = x0[c] + s * D[c]; Dhit[c] = D[c]; }",
                           "      for (int c = 0; c < 3; c++) { P[c] = x[c]; Dhit[c] = D[c]; }",
                           "twist_frame_hits or fourth_order"),
    "twist_hessian_dropped_zz": ("  H[1 * 9 + 2 * 3 + 2] = -k * k * (s * x + c * y);", "  H[1 * 9 + 2 * 3 + 2] = 0.0;",
                                 "twist_frame_hits"),
    # Riemannian illumination (pins in test_oracle_illum.py)
    "illum_euclidean_cosine": ("cosg = (n[0] * u[0] + n[1] * u[1] + n[2] * u[2]) / sqrt(nn);",
                               "cosg = (n[0] * u[0] + n[1] * u[1] + n[2] * u[2]);", "affine or radial",
                               "test_oracle_illum.py"),
    "illum_no_shadow": ("    if (blocked) lit = 0;\n", "", "flat", "test_oracle_illum.py"),
    "illum_gauss_newton_sign": ("      r1 -= Jc[1][c] * e[c];", "      r1 += Jc[1][c] * e[c];", "twist or radial",
                                "test_oracle_illum.py"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new, select = MUTANTS[name][:3]
    pins = MUTANTS[name][3] if len(MUTANTS[name]) > 3 else "test_oracle_pins.py"
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(so), str(mut), "-lm", "-lpthread"])
    env = dict(os.environ, RGEO_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins), "-k", select],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout + r.stderr
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
