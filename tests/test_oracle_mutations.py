"""Mutation check of the oracle's pins: plant one plausible mistake at a time
in a copy of the oracle source (a swapped weight, a dropped factor, a wrong
sign, a transposed operand, the paper's two misprints), build it, and require
that the pin tests fail.  Runs on the CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "spinsim_oracle.c")

MUTATIONS = {
    "cf4_weights_swapped": ("hb1[j] = wa * h1[j] + wb * h2[j];", "hb1[j] = wb * h1[j] + wa * h2[j];"),
    "cf4_node_sign": ("double t1 = t + 0.5 * (1.0 - 1.0 / r3) * dt;", "double t1 = t + 0.5 * (1.0 + 1.0 / r3) * dt;"),
    "cf4_exponential_order": ("mat_mul(n, E2, E1, u);", "mat_mul(n, E1, E2, u);"),
    "postmultiply_step": ("mat_mul(n, u, Ur, tmp);", "mat_mul(n, Ur, u, tmp);"),
    "paper_centre_misprint": ("T[1][1] = cos(Phi) * cexp(I * 2.0 * q / 3.0);", "T[1][1] = cos(Phi) * cexp(I * 4.0 * q);"),
    "paper_corner_misprint": ("T[0][2] = -(S * conj(eq6) * emiphi) * (S * conj(eq6) * emiphi);",
                              "T[0][2] = -(S * eq6 * emiphi) * (S * eq6 * emiphi);"),
    "dt_missing_in_z": ("double z = wz * dt / n;", "double z = wz / n;"),
    "residual_square_wrong": ("for (int i = 0; i < 3; i++) ap2[i][i] += 2.0;\n        mat_mul(3, ap2, a, s);\n        mat_copy(a, s);\n    }\n    mat_copy(E, a);",
                              "for (int i = 0; i < 3; i++) ap2[i][i] += 1.0;\n        mat_mul(3, ap2, a, s);\n        mat_copy(a, s);\n    }\n    mat_copy(E, a);"),
    "expm1_diag_factor": ("a[1][1] = expm1_i(th1) - 2.0 * S * S * cexp(I * th1);", "a[1][1] = expm1_i(th1) - S * S * cexp(I * th1);"),
    "frame_rotation_sign": ("w[1] = -wx * sin(a) + wy * cos(a);", "w[1] = wx * sin(a) + wy * cos(a);"),
    "frame_exit_sign": ("cplx ph = cexp(-I * m * w_r * p->dt_out);", "cplx ph = cexp(I * m * w_r * p->dt_out);"),
    "half_sigma_y_sign": ("cplx u01 = -I * s * (vx - I * vy);", "cplx u01 = -I * s * (vx + I * vy);"),
    "gaussian_width": ("exp(-(d * d) / (2.0 * wd * wd))", "exp(-(d * d) / (wd * wd))"),
    "sine_pulse_cosine": ("bz += f->pulse_amp_hz[p] * sin(2.0 * OR_PI * cyc);",
                          "bz += f->pulse_amp_hz[p] * cos(2.0 * OR_PI * cyc);"),
    "sine_pulse_half_period": ("bz += f->pulse_amp_hz[p] * sin(2.0 * OR_PI * cyc);",
                               "bz += f->pulse_amp_hz[p] * sin(OR_PI * cyc);"),
    "sine_pulse_window": ("if (cyc >= 0.0 && cyc < 1.0)", "if (cyc >= 0.0 && cyc < 0.5)"),
    "drive_y_cos": ("w[1] = 2.0 * OR_PI * f->drive_y_hz * sin(phase);", "w[1] = 2.0 * OR_PI * f->drive_y_hz * cos(phase);"),
    "tone_y_cos": ("w[1] += 2.0 * OR_PI * f->tone_y_hz[j] * sin(ph);", "w[1] += 2.0 * OR_PI * f->tone_y_hz[j] * cos(ph);"),
    "tone_phase_ignored": ("double ph = 2.0 * OR_PI * f->tone_hz[j] * t + f->tone_phase[j];",
                           "double ph = 2.0 * OR_PI * f->tone_hz[j] * t;"),
    "tones_dropped": ("for (int j = 0; j < f->n_tones && j < OR_MAX_TONES; j++) {",
                      "for (int j = 0; j < f->n_tones - 1 && j < OR_MAX_TONES; j++) {"),
    "su3_dxy_antisymmetric": ("G[7][i][j] = xy[i][j] + yx[i][j];", "G[7][i][j] = xy[i][j] - yx[i][j];"),
    "su3_pair2_single_angle": ("w[6] = u2 * cos(2.0 * a) + u3 * sin(2.0 * a);", "w[6] = u2 * cos(a) + u3 * sin(a);"),
    "qdrive_y_cos": ("u[2 * p + 1] = f->qd_on ? 2.0 * OR_PI * f->qd_y_hz[p] * sin(ph) : 0.0;",
                     "u[2 * p + 1] = f->qd_on ? 2.0 * OR_PI * f->qd_y_hz[p] * cos(ph) : 0.0;"),
    "su3_squaring_dropped": ("for (int q = 0; q < s; q++) {", "for (int q = 1; q < s; q++) {"),
    "jy_sign": ("J[1][0][1] = -I * r; J[1][1][0] = I * r;", "J[1][0][1] = I * r; J[1][1][0] = -I * r;"),
    "chain_transposed": ("s += U[i][j] * psi[j];", "s += U[j][i] * psi[j];"),
    "midpoint_node": ("field_in_frame(f, t + 0.5 * dt, t_ref, w_r, h);", "field_in_frame(f, t + dt, t_ref, w_r, h);"),
    "frame_midpoint": ("oracle_field_sample(f, t_prev + 0.5 * p->dt_out, wm);", "oracle_field_sample(f, t_prev, wm);"),
    "frame_off_ignored": ("if (!p->rotating_frame) return 0.0;", "if (0) return 0.0;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_detect_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", str(mutated), "-o", str(lib), "-lm"])
    env = dict(os.environ, SPINSIM_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_expm.py"),
                        os.path.join(ROOT, "tests", "test_oracle_dynamics.py"),
                        os.path.join(ROOT, "tests", "test_oracle_su3.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the oracle pins:\n{r.stdout[-2000:]}"
