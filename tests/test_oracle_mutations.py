"""The oracle pins have teeth: plant plausible mistakes in a copy of the oracle and
check that the pin suite (test_oracle_dynamics.py, test_oracle_models.py,
test_oracle_actions.py, test_oracle_randomization.py) fails on each.

Mistakes are planted only in a temporary copy of the oracle, on the CPU; the real
oracle is not modified. CPU only.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name: (text in mdg_oracle.c, planted mistake)
MUTATIONS = {
    "gyroscopic_sign": ("wdot[r] = (tau[r] - gyro[r]) / J[r];", "wdot[r] = (tau[r] + gyro[r]) / J[r];"),
    "semi_implicit_position": ("pn[r] = p[r] + dt * v[r];",
                               "pn[r] = p[r] + dt * (v[r] + dt * F[3 * j + r] / P->mass);"),
    "world_frame_rate": ("orc_quat_mul(q, dq, qn);", "orc_quat_mul(dq, q, qn);"),
    "full_angle_exp_map": ("double half = 0.5 * wnorm * dt;", "double half = wnorm * dt;"),
    "transposed_thrust_axis": ("double fw[3] = {R[2] * T, R[5] * T, R[8] * T - P->mass * P->g};",
                               "double fw[3] = {R[6] * T, R[7] * T, R[8] * T - P->mass * P->g};"),
    "drag_axis_coefficient": ("fb[2] = -P->c_z * omega_sum * vb[2];", "fb[2] = -P->c_xy * omega_sum * vb[2];"),
    "drag_not_rotated_back": (
        "for (int r = 0; r < 3; ++r) fw[r] += R[3 * r + 0] * fb[0] + R[3 * r + 1] * fb[1] + R[3 * r + 2] * fb[2];",
        "for (int r = 0; r < 3; ++r) fw[r] += R[r + 0] * fb[0] + R[r + 3] * fb[1] + R[r + 6] * fb[2];"),
    "ground_effect_not_squared": ("fw[2] += P->c_gnd * T * r * r;", "fw[2] += P->c_gnd * T * r;"),
    "ground_effect_ungated": ("if (fabs(rpy[0]) < ORC_PI / 2 && fabs(rpy[1]) < ORC_PI / 2) {", "if (1) {"),
    "downwash_dz_sign": ("double dz = xi[2] - xj[2];", "double dz = xj[2] - xi[2];"),
    "downwash_gaussian_half": ("fw[2] -= alpha * exp(-0.5 * dxy * dxy / b2);",
                               "fw[2] -= alpha * exp(-dxy * dxy / b2);"),
    "yaw_torque_sign": ("tau[2] = P->km * (-n2[0] + n2[1] - n2[2] + n2[3]);",
                        "tau[2] = P->km * (n2[0] - n2[1] + n2[2] - n2[3]);"),
    "roll_torque_pairing": ("tau[0] = l * (F[0] + F[1] - F[2] - F[3]);", "tau[0] = l * (F[0] - F[1] - F[2] + F[3]);"),
    "inertia_index": ("double Jw[3] = {J[0] * w[0], J[1] * w[1], J[2] * w[2]};",
                      "double Jw[3] = {J[0] * w[0], J[2] * w[1], J[1] * w[2]};"),
    "pid_derivative_sign": (
        "a[r] = P->pos_kp[r] * ep[r] + P->pos_ki[r] * I + P->pos_kd[r] * (v_t[r] - v[r]);",
        "a[r] = P->pos_kp[r] * ep[r] + P->pos_ki[r] * I + P->pos_kd[r] * (v[r] - v_t[r]);"),
    "pid_roll_target_sign": ("double phi_t = (a[0] * sin(psi_t) - a[1] * cos(psi_t)) / P->g;",
                             "double phi_t = (a[0] * sin(psi_t) + a[1] * cos(psi_t)) / P->g;"),
    "pitch_extraction": ("double sp = 2.0 * (w * y - z * x);", "double sp = 2.0 * (w * y + z * x);"),
    "knn_tie_order": ("while (pos > 0 && d2 < bestd[pos - 1]) --pos;", "while (pos > 0 && d2 <= bestd[pos - 1]) --pos;"),
    "no_renormalisation": ("for (int r = 0; r < 4; ++r) o[3 + r] = qn[r] / qnorm;",
                           "for (int r = 0; r < 4; ++r) o[3 + r] = qn[r];"),
    "rk4_third_stage_from_k1": ("for (size_t i = 0; i < m; ++i) xs[i] = x_in[i] + 0.5 * dt * k2[i];",
                                "for (size_t i = 0; i < m; ++i) xs[i] = x_in[i] + 0.5 * dt * k1[i];"),
    "rk4_weights": ("dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i])",
                    "dt / 6.0 * (2.0 * k1[i] + k2[i] + 2.0 * k3[i] + k4[i])"),
    "rk4_quaternion_rate_sign": ("for (int r = 0; r < 4; ++r) d[3 + r] = 0.5 * qd[r];",
                                 "for (int r = 0; r < 4; ++r) d[3 + r] = -0.5 * qd[r];"),
    "plus_roll_pair": ("tau[0] = P->arm * (F[1] - F[3]);", "tau[0] = P->arm * (F[0] - F[2]);"),
    "plus_allocation_row": ("{{1, 1, 1, 1}, {0, L, 0, -L}, {-L, 0, L, 0}, {-r, r, -r, r}}",
                            "{{1, 1, 1, 1}, {L, 0, -L, 0}, {-L, 0, L, 0}, {-r, r, -r, r}}"),
    "race_gain_ratio": ("P->att_kp[r] = cf.att_kp[r] * ratio[r];", "P->att_kp[r] = cf.att_kp[r];"),
    "rotor_height_sign": ("double zi = xj[2] + R[6] * ri[0] + R[7] * ri[1] + R[8] * ri[2];",
                          "double zi = xj[2] - R[6] * ri[0] - R[7] * ri[1] - R[8] * ri[2];"),
    "rotor_height_transposed": ("double zi = xj[2] + R[6] * ri[0] + R[7] * ri[1] + R[8] * ri[2];",
                                "double zi = xj[2] + R[2] * ri[0] + R[5] * ri[1] + R[8] * ri[2];"),
    "rotor_height_at_com": ("double r = P->prop_radius / (4.0 * fmax(zi, P->h_clip));",
                            "double r = P->prop_radius / (4.0 * fmax(xj[2], P->h_clip));"),
    "rotor_positions_swapped": ("r[0] = l * xs[i];", "r[0] = l * ys[i];"),
    "vel_world_frame": (
        "for (int r = 0; r < 3; ++r) v_t[r] = R[3 * r] * act[0] + R[3 * r + 1] * act[1] + R[3 * r + 2] * act[2];",
        "for (int r = 0; r < 3; ++r) v_t[r] = act[r];"),
    "attitude_roll_pitch_swap": ("att[0] = act[1];", "att[0] = act[2];"),
    "normalized_upper_slope": ("return a <= 0.0 ? hover * (1.0 + a) : hover + (maxrpm - hover) * a;",
                               "return a <= 0.0 ? hover * (1.0 + a) : hover * (1.0 + a);"),
    "yaw_rate_sign": ("const double w_t[3] = {0.0, 0.0, act[3]};", "const double w_t[3] = {0.0, 0.0, -act[3]};"),
    "dsl_rate_limit_dropped": ("const double s = n > lim ? lim / n : 1.0;", "const double s = 1.0;"),
    "dsl_yaw_limit_sign": ("if (dy < -ly) dy = -ly;", "if (dy < -ly) dy = ly;"),
    "feed_forward_dropped": ("a[r] += a_ff[r];", "a[r] += 0.0 * a_ff[r];"),
    "dsl_setpoint_unused": ("        tgt = sp;\n", "        tgt = wp;\n"),
    "dr_mass_dropped": ("    Pe->mass *= dr[ORC_DR_MASS];\n", "\n"),
    "wind_drag_sign": ("const double vr[3] = {v_w[0] - v[0], v_w[1] - v[1], v_w[2] - v[2]};",
                       "const double vr[3] = {v[0] - v_w[0], v[1] - v_w[1], v[2] - v_w[2]};"),
    "lag_discretization": ("*m = c + (*m - c) * lag;", "*m = c + (*m - c) * (1.0 - lag);"),
    "latency_newest": ("a = h0 + (size_t)row[ORC_DR_DELAY] * hs;", "a = h0;"),
    "dryden_noise_scale": ("sqrt(1.0 - alpha * alpha) * xi[r]", "sqrt(1.0 - alpha) * xi[r]"),
    "gust_envelope": ("sin(ORC_PI * ws[3])", "sin(2.0 * ORC_PI * ws[3])"),
    "sinusoid_phase": ("F_dir[0] += A * sin(w * t);", "F_dir[0] += A * cos(w * t);"),
    "motor_bias_dropped": ("c *= row[ORC_DR_BIAS + i];", "c *= 1.0;"),
    "arm_factor_to_inertia": ("    Pe->arm *= dr[ORC_DR_ARM];\n", "    Pe->Jxx *= dr[ORC_DR_ARM];\n"),
    "sensor_delay_ignored": ("const int delayed = row && x_last && K > 0 && row[ORC_DR_OBS_DELAY] == 1.0;",
                             "const int delayed = 0;"),
    "noise_rpy_channel": ("o[7 + r] += row[ORC_DR_NOISE_RPY] * xi[3 + r];", "o[3 + r] += row[ORC_DR_NOISE_RPY] * xi[3 + r];"),
    "reset_xyz_euler_order": ("orc_quat_mul(qz, qy, qzy);", "orc_quat_mul(qy, qz, qzy);"),
    "reset_full_angle": ("const double qx[4] = {cos(0.5 * roll), sin(0.5 * roll), 0.0, 0.0};",
                         "const double qx[4] = {cos(roll), sin(roll), 0.0, 0.0};"),
    "reset_velocity_range": ("x[7 + k] = r[2] * u[6 + k];", "x[7 + k] = r[2] * (0.5 + 0.5 * u[6 + k]);"),
    "bias_sigma_group": ("b[2 * m] = sigma[(2 * m) / 3] * rho * cos(2.0 * ORC_PI * u2);",
                         "b[2 * m] = sigma[m / 3] * rho * cos(2.0 * ORC_PI * u2);"),
    "bias_rate_channel": ("o[13 + r] += bb[9 + r];", "o[13 + r] += bb[6 + r];"),
}


# planted in oracle/mlp.py, caught by tests/test_oracle_mlp.py
MLP_MUTATIONS = {
    "silu_grad_sign": ("return s * (1.0 + z * (1.0 - s))", "return s * (1.0 - z * (1.0 - s))"),
    "mse_grad_factor": ("dz = q(2.0 * (y - t) / y.size)", "dz = q((y - t) / y.size)"),
    "adam_bias_correction": ("c1, c2 = 1.0 - b1 ** step, 1.0 - b2 ** step", "c1, c2 = 1.0, 1.0 - b2 ** step"),
    "backprop_through_weights": ("dz = q((dz @ Wl) * silu_grad(zs[l - 1]))", "dz = q((dz @ Wl) * silu(zs[l - 1]))"),
    "bf16_tie_rounding": ("rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "rounded = ((u + 0x8000) >> 16) << 16"),
}


@pytest.fixture(scope="module")
def oracle_source():
    with open(os.path.join(ROOT, "oracle", "mdg_oracle.c")) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, oracle_source, tmp_path):
    before, after = MUTATIONS[name]
    assert oracle_source.count(before) == 1, f"mutation site of {name} not found exactly once"
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle", ignore=shutil.ignore_patterns("_build"))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests",
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py"))
    # the pins read their inputs from the package's generators (Python only)
    shutil.copytree(os.path.join(ROOT, "paper_2606_08039_gb300"), tmp_path / "paper_2606_08039_gb300",
                    ignore=shutil.ignore_patterns("__pycache__", "csrc", "_build", "*.so"))
    (tmp_path / "oracle" / "mdg_oracle.c").write_text(oracle_source.replace(before, after))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_dynamics.py", "tests/test_oracle_models.py",
                        "tests/test_oracle_actions.py", "tests/test_oracle_randomization.py", "-q", "-x", "-p",
                        "no:cacheprovider"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 1, f"planted mistake {name} was not caught:\n{r.stdout[-2000:]}"


# planted in oracle/camera.py, caught by tests/test_oracle_camera.py
CAMERA_MUTATIONS = {
    "camera_fov_horizontal": ("    nx = c * th * W / H\n", "    nx = c * th\n"),
    "camera_euclidean_depth": ("depth = np.where(np.isfinite(t_best), t_best * (dn @ fwd), np.inf)",
                               "depth = np.where(np.isfinite(t_best), t_best, np.inf)"),
    "camera_light_sign": ("np.maximum(0.0, n @ LIGHT)", "np.maximum(0.0, -(n @ LIGHT))"),
    "camera_own_drone_drawn": ("        if k == j:\n            continue\n", ""),
    "camera_segment_id": ("seg = np.where(better, 1 + first_index + k, seg)", "seg = np.where(better, first_index + k, seg)"),
}


@pytest.mark.parametrize("name", sorted(CAMERA_MUTATIONS))
def test_planted_camera_mistake_is_caught(name, tmp_path):
    before, after = CAMERA_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "camera.py")).read()
    assert src.count(before) == 1, f"mutation site of {name} not found exactly once"
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle", ignore=shutil.ignore_patterns("_build"))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests",
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py"))
    (tmp_path / "oracle" / "camera.py").write_text(src.replace(before, after))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_camera.py", "-q", "-x", "-p",
                        "no:cacheprovider"], cwd=tmp_path, capture_output=True, text=True, timeout=300)
    assert r.returncode == 1, f"planted mistake {name} was not caught:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", sorted(MLP_MUTATIONS))
def test_planted_mlp_mistake_is_caught(name, tmp_path):
    before, after = MLP_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "mlp.py")).read()
    assert src.count(before) == 1, f"mutation site of {name} not found exactly once"
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle", ignore=shutil.ignore_patterns("_build"))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests",
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py"))
    (tmp_path / "oracle" / "mlp.py").write_text(src.replace(before, after))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_mlp.py", "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=tmp_path, capture_output=True, text=True, timeout=300)
    assert r.returncode == 1, f"planted mistake {name} was not caught:\n{r.stdout[-2000:]}"
