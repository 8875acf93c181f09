/*
 * FP64 CPU oracle of the batched Crazyflie 2.x dynamics step (MuJoCo-Drones-Gym,
 * Section 3.1 "Quadrotor Dynamics", Section 3.2 "Physics Modes", Section 4.2
 * "Control").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the correctness reference that the
 * test suite, the smoke check and the benchmark's CPU-baseline leg compare the
 * CUDA library against. The product path never links, loads or calls it, and it
 * shares no code, header, constant table or helper with the CUDA library.
 *
 * It is written to be read against the paper, not to be fast: every drone of an
 * environment is handled by plain loops in double precision, each step in the
 * order the paper states it. Where the paper is silent the reading taken is named
 * in the comment beside the code.
 *
 * Parity pins: every function here is checked by tests that do not re-derive it
 * (closed forms, invariants, special cases, brute force); see the tests named
 * test_oracle_*.py.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -o liboracle.so mdg_oracle.c -lm
 * (-ffp-contract=off: every product and sum rounds as written, the same on x86 and Arm.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* Physics-mode bits (Table "Physics modes": ground effect, drag, downwash). */
#define ORC_GND 1
#define ORC_DRAG 2
#define ORC_DW 4

/* Action types (Table "Action types"): raw RPM or an absolute PID waypoint. */
#define ORC_ACT_RPM 0
#define ORC_ACT_PID 1
#define ORC_ACT_RPM_NORM 3
#define ORC_ACT_ONE_D_RPM 4
#define ORC_ACT_VEL 5
#define ORC_ACT_ATTITUDE 6

/* Rotor layouts (Section 3.1.2): X configuration (CF2X, RACE) or + configuration (CF2P). */
#define ORC_FRAME_X 0
#define ORC_FRAME_P 1

/* Integrators (Table "Physics modes"): the explicit Euler of the DYN mode, or classical
 * fourth-order Runge-Kutta (the MuJoCo modes integrate with RK4). */
#define ORC_EULER 0
#define ORC_RK4 1

/* Heights at which Eq. ground is evaluated: the centre of mass for all four rotors (h from
 * p_z, as printed), or each rotor's own height (a variant: rotor i adds
 * C_gnd k_f n_i^2 (r_p/(4 h_i))^2, h_i = max(p_z + (R r_i)_z, h_clip), r_i its body
 * position). */
#define ORC_GND_COM 0
#define ORC_GND_ROTOR 1

/* Controllers (Section 4.2.1): PIDControl, or DSLPIDControl (retuned gains, halved
 * integral clamps, rate-limited position and yaw setpoints, feed-forward acceleration). */
#define ORC_CTRL_PID 0
#define ORC_CTRL_DSL 1

/* Domain randomization (Section 3.5, Table "Recommended domain-randomization ranges")
 * and wind (Section 3.5, "Wind and turbulence"): one row of ORC_DR_PARAMS values per
 * environment. Multiplicative factors scale the model the physics integrates; the
 * controller keeps the nominal model (it does not know the draw). */
#define ORC_DR_PARAMS 40
#define ORC_DR_MASS 0      /* x m */
#define ORC_DR_J 1         /* x Jxx, Jyy, Jzz (1..3) */
#define ORC_DR_ARM 4       /* x L */
#define ORC_DR_KF 5        /* x k_f */
#define ORC_DR_KM 6        /* x k_m */
#define ORC_DR_CXY 7       /* x c_xy */
#define ORC_DR_CZ 8        /* x c_z */
#define ORC_DR_CGND 9      /* x C_gnd */
#define ORC_DR_C1 10       /* x downwash C1 */
#define ORC_DR_MAXRPM 11   /* x MAX_RPM (the motors' saturation) */
#define ORC_DR_BIAS 12     /* per-motor speed bias (12..15) */
#define ORC_DR_G 16        /* x g */
#define ORC_DR_TAU 17      /* motor lag time constant [s], 0 = none */
#define ORC_DR_DELAY 18    /* action latency [control steps], a whole number */
#define ORC_DR_WIND 19     /* wind model bits: CONSTANT 1, GUST 2, DRYDEN 4, SINUSOIDAL 8 */
#define ORC_DR_VWIND 20    /* steady wind velocity [m/s], world frame (20..22) */
#define ORC_DR_KDRAG 23    /* 1/2 rho C_d A [kg/m] of the quadratic wind drag */
#define ORC_DR_GUST_P 24   /* gust trigger probability per control step */
#define ORC_DR_GUST_A 25   /* gust amplitude [N] */
#define ORC_DR_GUST_T 26   /* gust duration [s] */
#define ORC_DR_DRY_SIGMA 27 /* Dryden turbulence intensity [m/s] */
#define ORC_DR_DRY_V 28    /* Dryden airspeed V [m/s] */
#define ORC_DR_SIN_A 29    /* sinusoidal amplitude A [N] */
#define ORC_DR_SIN_W 30    /* sinusoidal angular frequency [rad/s] */
#define ORC_DR_DRY_H 31    /* Dryden reference altitude h [m] */
#define ORC_DR_NOISE_P 32  /* observation noise: position sigma [m] */
#define ORC_DR_NOISE_V 33  /* velocity sigma [m/s] */
#define ORC_DR_NOISE_RPY 34 /* roll, pitch, yaw sigma [rad] */
#define ORC_DR_NOISE_W 35  /* gyro (body rate) sigma [rad/s] */
#define ORC_DR_OBS_DELAY 36 /* sensor latency [control steps]: 0 or 1 */
#define ORC_WIND_CONSTANT 1
#define ORC_WIND_GUST 2
#define ORC_WIND_DRYDEN 4
#define ORC_WIND_SINUSOIDAL 8
#define ORC_WIND_STATE 8   /* per environment: Dryden x (3), gust phase s (-1 idle), gust direction (3), steps */
#define ORC_STREAM_WIND 21 /* random stream of the wind draws */
#define ORC_STREAM_OBS 22  /* random stream of the observation noise */
#define ORC_STREAM_INIT 23 /* random stream of the per-episode initial states */
#define ORC_STREAM_BIAS 24 /* random stream of the per-episode observation bias */

/* Model parameters. Field order is the oracle's own; the Python side of the
 * oracle mirrors it. */
typedef struct {
    /* Table "Drone model parameters", CF2X column. */
    double mass, arm, thrust2weight, Jxx, Jyy, Jzz, kf, km, prop_radius;
    double g;
    /* Eq. ground, Eq. drag, Eq. downwash coefficients. */
    double c_gnd, h_clip, c_xy, c_z;
    double dw_c1, dw_c2, dw_c3, dw_max_xy, dw_dz_min;
    /* Table "Default PIDControl gains". */
    double pos_kp[3], pos_ki[3], pos_kd[3], pos_iclamp;
    double att_kp[3], att_ki[3], att_kd[3], att_iclamp;
    double dt_sim, dt_ctrl;
    /* DSLPIDControl's setpoint rate limits (m/s, rad/s) */
    double sp_rate_pos, sp_rate_yaw;
    int32_t frame;      /* ORC_FRAME_X / ORC_FRAME_P */
    int32_t integrator; /* ORC_EULER / ORC_RK4 */
    int32_t gnd_heights; /* ORC_GND_COM / ORC_GND_ROTOR */
    int32_t controller;  /* ORC_CTRL_PID / ORC_CTRL_DSL */
} orc_params;

int orc_params_size(void) { return (int)sizeof(orc_params); }

/* Section 3.3: HOVER_RPM = sqrt(m g / (4 k_f)). */
double orc_hover_rpm(const orc_params* P) { return sqrt(P->mass * P->g / (4.0 * P->kf)); }

/* Section 3.3: MAX_RPM from (m, g, k_f, T/W): the four rotors at MAX_RPM give
 * thrust2weight times the weight, 4 k_f MAX_RPM^2 = (T/W) m g. */
double orc_max_rpm(const orc_params* P)
{
    return sqrt(P->thrust2weight * P->mass * P->g / (4.0 * P->kf));
}

/* Default constants. Table "Drone model parameters" (CF2X), the downwash
 * coefficients of Eq. downwash and the gains of Table "Default PIDControl gains"
 * are printed in the paper. g, C_gnd, c_xy, c_z are not printed: g is MuJoCo's
 * default gravity, the three aerodynamic coefficients are documented defaults.
 * h_clip is "derived from the propeller radius and the model's maximum thrust"
 * (Section 3.1.3): it is the height at which the ground-effect increment at hover
 * thrust equals the spare thrust MAX_THRUST - m g, i.e.
 * C_gnd m g (r_p/(4 h))^2 = (T/W - 1) m g. */
void orc_params_cf2x(orc_params* P)
{
    memset(P, 0, sizeof(*P));
    P->mass = 0.027;
    P->arm = 0.0397;
    P->thrust2weight = 2.25;
    P->Jxx = 1.4e-5;
    P->Jyy = 1.4e-5;
    P->Jzz = 2.17e-5;
    P->kf = 3.16e-10;
    P->km = 7.94e-12;
    P->prop_radius = 0.02325;
    P->g = 9.81;
    P->c_gnd = 11.36859;
    P->h_clip = 0.25 * P->prop_radius * sqrt(P->c_gnd / (P->thrust2weight - 1.0));
    P->c_xy = 9.1785e-7;
    P->c_z = 10.311e-7;
    P->dw_c1 = 2267.18;
    P->dw_c2 = 0.16;
    P->dw_c3 = -0.11;
    P->dw_max_xy = 10.0;
    P->dw_dz_min = 0.0;
    P->pos_kp[0] = 0.4; P->pos_kp[1] = 0.4; P->pos_kp[2] = 1.0;
    P->pos_ki[0] = 0.01; P->pos_ki[1] = 0.01; P->pos_ki[2] = 0.01;
    P->pos_kd[0] = 0.9; P->pos_kd[1] = 0.9; P->pos_kd[2] = 2.0;
    P->pos_iclamp = 2.0;
    P->att_kp[0] = 2e-3; P->att_kp[1] = 2e-3; P->att_kp[2] = 1e-3;
    P->att_ki[0] = 0.0; P->att_ki[1] = 0.0; P->att_ki[2] = 1e-4;
    P->att_kd[0] = 5e-4; P->att_kd[1] = 5e-4; P->att_kd[2] = 2e-4;
    P->att_iclamp = 0.5;
    P->dt_sim = 1.0 / 240.0;
    P->dt_ctrl = 1.0 / 48.0;
    P->frame = ORC_FRAME_X;
    P->integrator = ORC_EULER;
    P->gnd_heights = ORC_GND_COM;
    P->sp_rate_pos = 2.0;
    P->sp_rate_yaw = ORC_PI;
    P->controller = ORC_CTRL_PID;
}

/* CF2P: the CF2X parameters (Table "Drone model parameters" lists one column for both)
 * with the + rotor layout. */
void orc_params_cf2p(orc_params* P)
{
    orc_params_cf2x(P);
    P->frame = ORC_FRAME_P;
}

/* RACE: the RACE column of Table "Drone model parameters". Not printed for RACE, and
 * read here: the aerodynamic coefficients (C_gnd, c_xy, c_z, C1..C3) keep their CF2.x
 * values, h_clip follows the same derivation from r_p and T/W, the position-loop gains
 * (which command accelerations; the thrust T = m |a*| scales with the mass) are kept, and
 * the attitude-loop gains (which command torques) are scaled per axis by the inertia ratio
 * J_RACE / J_CF2 so that the angular-acceleration response matches the Crazyflie's. */
void orc_params_race(orc_params* P)
{
    orc_params cf;
    orc_params_cf2x(&cf);
    *P = cf;
    P->mass = 0.25;
    P->arm = 0.125;
    P->thrust2weight = 4.0;
    P->Jxx = 4.86e-4;
    P->Jyy = 4.86e-4;
    P->Jzz = 8.80e-4;
    P->kf = 1.28e-8;
    P->km = 5.96e-10;
    P->prop_radius = 0.0635;
    P->h_clip = 0.25 * P->prop_radius * sqrt(P->c_gnd / (P->thrust2weight - 1.0));
    const double ratio[3] = {P->Jxx / cf.Jxx, P->Jyy / cf.Jyy, P->Jzz / cf.Jzz};
    for (int r = 0; r < 3; ++r) {
        P->att_kp[r] = cf.att_kp[r] * ratio[r];
        P->att_ki[r] = cf.att_ki[r] * ratio[r];
        P->att_kd[r] = cf.att_kd[r] * ratio[r];
    }
}

/* ---- quaternion helpers; q = [w, x, y, z], body-to-world (Section 3.1.1) ---- */

/* Hamilton product a (x) b. */
void orc_quat_mul(const double a[4], const double b[4], double out[4])
{
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    out[0] = w; out[1] = x; out[2] = y; out[3] = z;
}

/* Rotation matrix R (row-major 3x3) of a unit quaternion: world = R * body. */
void orc_rotation(const double q[4], double R[9])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Roll, pitch, yaw (ZYX convention, R = Rz(yaw) Ry(pitch) Rx(roll)), the eta of
 * the KIN observation (Section 3.4.4). */
void orc_rpy(const double q[4], double rpy[3])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    double sp = 2.0 * (w * y - z * x);
    if (sp > 1.0) sp = 1.0;
    if (sp < -1.0) sp = -1.0;
    rpy[0] = atan2(2.0 * (w * x + y * z), 1.0 - 2.0 * (x * x + y * y));
    rpy[1] = asin(sp);
    rpy[2] = atan2(2.0 * (w * z + x * y), 1.0 - 2.0 * (y * y + z * z));
}

/* DSLPIDControl (Section 4.2.1): "retunes the position and attitude gains" (not printed),
 * "halves the integral clamps" and rate-limits the position (2.0 m/s) and yaw (pi rad/s)
 * setpoints. Reading for the gains: each loop is tuned as a second-order system,
 * x'' + Kd x' + Kp x = 0 for the position loop (the PID commands an acceleration) and
 * J x'' + Kd x' + Kp x = 0 for the attitude loop (it commands a torque), with natural
 * frequency w_n and damping z: Kp = w_n^2, Kd = 2 z w_n (position; w_n = 1.5, 1.5, 2.0 rad/s,
 * z = 0.8, 0.8, 1.0, Ki = 0.05) and Kp = J w_n^2, Kd = 2 z w_n J (attitude; w_n = 20, 20,
 * 10 rad/s, z = 0.9, Ki = J (0, 0, 5)), the model's own J. The clamps are half of P's. */
void orc_controller_dsl(orc_params* P)
{
    const double wp[3] = {1.5, 1.5, 2.0}, zp[3] = {0.8, 0.8, 1.0};
    const double wa[3] = {20.0, 20.0, 10.0}, za = 0.9, kia[3] = {0.0, 0.0, 5.0};
    const double J[3] = {P->Jxx, P->Jyy, P->Jzz};
    for (int r = 0; r < 3; ++r) {
        P->pos_kp[r] = wp[r] * wp[r];
        P->pos_kd[r] = 2.0 * zp[r] * wp[r];
        P->pos_ki[r] = 0.05;
        P->att_kp[r] = J[r] * wa[r] * wa[r];
        P->att_kd[r] = 2.0 * za * wa[r] * J[r];
        P->att_ki[r] = J[r] * kia[r];
    }
    P->pos_iclamp *= 0.5;
    P->att_iclamp *= 0.5;
    P->controller = ORC_CTRL_DSL;
}

/* ---- forces: Eq. motor, Eq. ground, Eq. drag, Eq. downwash ---- */

/* Eq. motor with the X-configuration mixing (Section 3.1.2): per-rotor thrust
 * F_i = k_f n_i^2, collective thrust T = sum F_i, body torques
 * tau_x = L/sqrt2 (F0 + F1 - F2 - F3), tau_y = L/sqrt2 (-F0 + F1 + F2 - F3) and
 * the yaw torque from the alternating reaction torques (-1)^{m_i} k_m n_i^2,
 * read as m = (1, 0, 1, 0): tau_z = k_m (-n0^2 + n1^2 - n2^2 + n3^2).
 * n is in RPM and k_f, k_m are per RPM^2 (HOVER_RPM with the printed k_f is
 * about 14476, an RPM figure). */
void orc_motor(const orc_params* P, const double rpm[4], double* T, double tau[3])
{
    double F[4], n2[4];
    for (int i = 0; i < 4; ++i) {
        n2[i] = rpm[i] * rpm[i];
        F[i] = P->kf * n2[i];
    }
    *T = F[0] + F[1] + F[2] + F[3];
    if (P->frame == ORC_FRAME_P) {
        /* + configuration: "the L/sqrt2 factor replaced by L on a different pair of
         * motors". Read as the X layout turned by 45 degrees: the X torques place rotor i
         * at (x, y) = L/sqrt2 ((+,+), (-,+), (-,-), (+,-)) (tau_x = sum y_i F_i,
         * tau_y = -sum x_i F_i); turned by 45 degrees the rotors sit at L (+x, +y, -x, -y),
         * so tau_x = L (F1 - F3), tau_y = L (F2 - F0); the yaw signs are unchanged. */
        tau[0] = P->arm * (F[1] - F[3]);
        tau[1] = P->arm * (F[2] - F[0]);
    } else {
        const double l = P->arm / sqrt(2.0);
        tau[0] = l * (F[0] + F[1] - F[2] - F[3]);
        tau[1] = l * (-F[0] + F[1] + F[2] - F[3]);
    }
    tau[2] = P->km * (-n2[0] + n2[1] - n2[2] + n2[3]);
}

/* Body-frame position of rotor i (z = 0). With tau = sum_i r_i x (0, 0, F_i), i.e.
 * tau_x = sum_i y_i F_i and tau_y = -sum_i x_i F_i, the torque equations of Section 3.1.2
 * place the X layout's rotors at L/sqrt2 (+,+), (-,+), (-,-), (+,-) and the + layout's at
 * L (+x, +y, -x, -y) (orc_motor). */
void orc_rotor_position(const orc_params* P, int i, double r[3])
{
    static const double xs[4] = {1.0, -1.0, -1.0, 1.0}, ys[4] = {1.0, 1.0, -1.0, -1.0};
    static const double xp[4] = {1.0, 0.0, -1.0, 0.0}, yp[4] = {0.0, 1.0, 0.0, -1.0};
    if (P->frame == ORC_FRAME_P) {
        r[0] = P->arm * xp[i];
        r[1] = P->arm * yp[i];
    } else {
        const double l = P->arm / sqrt(2.0);
        r[0] = l * xs[i];
        r[1] = l * ys[i];
    }
    r[2] = 0.0;
}

/* World-frame force (gravity included) and body-frame torque on every drone of
 * one environment of N drones. x is [N][13] = p(3) q(4) v(3) omega(3), omega in
 * the body frame; rpm is [N][4]. All drones read the same state snapshot x. */
void orc_env_forces(const orc_params* P, int N, const double* x, const double* rpm, int flags,
                    const double* f_ext, double* F, double* tau)
{
    for (int j = 0; j < N; ++j) {
        const double* xj = x + 13 * j;
        const double* q = xj + 3;
        const double* v = xj + 7;
        double T, R[9];
        orc_motor(P, rpm + 4 * j, &T, tau + 3 * j);
        orc_rotation(q, R);
        /* thrust along the body z axis, rotated to the world frame, and gravity */
        double fw[3] = {R[2] * T, R[5] * T, R[8] * T - P->mass * P->g};

        if (flags & ORC_GND) {
            /* Eq. ground: C_gnd * sum_i k_f n_i^2 * (r_p/(4h))^2, h = max(p_z, h_clip),
             * applied along world +z, gated on |roll|, |pitch| < pi/2. With per-rotor
             * heights, h_i = max(p_z + (R r_i)_z, h_clip) for rotor i. */
            double rpy[3];
            orc_rpy(q, rpy);
            if (fabs(rpy[0]) < ORC_PI / 2 && fabs(rpy[1]) < ORC_PI / 2) {
                if (P->gnd_heights == ORC_GND_ROTOR) {
                    const double* n = rpm + 4 * j;
                    for (int i = 0; i < 4; ++i) {
                        double ri[3];
                        orc_rotor_position(P, i, ri);
                        double zi = xj[2] + R[6] * ri[0] + R[7] * ri[1] + R[8] * ri[2];
                        double r = P->prop_radius / (4.0 * fmax(zi, P->h_clip));
                        fw[2] += P->c_gnd * P->kf * n[i] * n[i] * r * r;
                    }
                } else {
                    double h = fmax(xj[2], P->h_clip);
                    double r = P->prop_radius / (4.0 * h);
                    fw[2] += P->c_gnd * T * r * r;
                }
            }
        }
        if (flags & ORC_DRAG) {
            /* Eq. drag: F_body = -diag(c_xy, c_xy, c_z) (sum_i 2 pi n_i / 60) v_body,
             * v_body = R^T v, rotated back to the world frame by R. */
            const double* n = rpm + 4 * j;
            double omega_sum = 0.0;
            for (int i = 0; i < 4; ++i) omega_sum += 2.0 * ORC_PI * n[i] / 60.0;
            double vb[3], fb[3];
            for (int r = 0; r < 3; ++r) vb[r] = R[0 + r] * v[0] + R[3 + r] * v[1] + R[6 + r] * v[2];
            fb[0] = -P->c_xy * omega_sum * vb[0];
            fb[1] = -P->c_xy * omega_sum * vb[1];
            fb[2] = -P->c_z * omega_sum * vb[2];
            for (int r = 0; r < 3; ++r) fw[r] += R[3 * r + 0] * fb[0] + R[3 * r + 1] * fb[1] + R[3 * r + 2] * fb[2];
        }
        if (flags & ORC_DW) {
            /* Eq. downwash: every drone i strictly above j (dz > max(0, dz_min)) with
             * lateral separation dxy < dw_max_xy pushes j down by
             * alpha exp(-1/2 (dxy/beta)^2), alpha = C1 (r_p/(4 dz))^2, beta = C2 dz + C3.
             * beta^2 is floored at 1e-12 so that beta = 0 (dz = -C3/C2) stays finite. */
            const double dz_min = fmax(0.0, P->dw_dz_min);
            for (int i = 0; i < N; ++i) {
                if (i == j) continue;
                const double* xi = x + 13 * i;
                double dz = xi[2] - xj[2];
                if (!(dz > dz_min)) continue;
                double dxy = hypot(xi[0] - xj[0], xi[1] - xj[1]);
                if (!(dxy < P->dw_max_xy)) continue;
                double r = P->prop_radius / (4.0 * dz);
                double alpha = P->dw_c1 * r * r;
                double beta = P->dw_c2 * dz + P->dw_c3;
                double b2 = fmax(beta * beta, 1e-12);
                fw[2] -= alpha * exp(-0.5 * dxy * dxy / b2);
            }
        }
        if (f_ext) {
            /* an external world-frame force on the drone (wind; domain randomization) */
            for (int r = 0; r < 3; ++r) fw[r] += f_ext[3 * j + r];
        }
        F[3 * j + 0] = fw[0];
        F[3 * j + 1] = fw[1];
        F[3 * j + 2] = fw[2];
    }
}

/* Rotational Newton-Euler in the body frame: omega_dot = J^-1 (tau - omega x (J omega)). */
static void orc_angular_accel(const double J[3], const double tau[3], const double w[3], double wdot[3])
{
    double Jw[3] = {J[0] * w[0], J[1] * w[1], J[2] * w[2]};
    double gyro[3] = {w[1] * Jw[2] - w[2] * Jw[1], w[2] * Jw[0] - w[0] * Jw[2], w[0] * Jw[1] - w[1] * Jw[0]};
    for (int r = 0; r < 3; ++r) wdot[r] = (tau[r] - gyro[r]) / J[r];
}

/* One physics substep of length dt for one environment (Section 3.2, DYN mode,
 * "explicit Euler", plus the closed-form exponential map of _integrateQ).
 * Reading: forward Euler — p uses the old v, v the old acceleration, omega the
 * old angular acceleration, and q is advanced with the old omega. Newton-Euler:
 * a = F/m, omega_dot = J^-1 (tau - omega x (J omega)), omega in the body frame.
 * The exponential map is q+ = q (x) [cos(|w| dt/2), sin(|w| dt/2) w/|w|] (the
 * norm-preserving reading of the printed map with Lambda the half quaternion-product
 * matrix; a body-frame rate multiplies on the right), then q+ is renormalised. */
void orc_substep(const orc_params* P, int N, const double* x_in, const double* rpm, int flags,
                 const double* f_ext, double dt, double* x_out)
{
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double* tau = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    orc_env_forces(P, N, x_in, rpm, flags, f_ext, F, tau);
    const double J[3] = {P->Jxx, P->Jyy, P->Jzz};
    for (int j = 0; j < N; ++j) {
        const double* s = x_in + 13 * j;
        double* o = x_out + 13 * j;
        const double* p = s;
        const double* q = s + 3;
        const double* v = s + 7;
        const double* w = s + 10;
        double wdot[3];
        orc_angular_accel(J, tau + 3 * j, w, wdot);
        double pn[3], vn[3], wn[3], qn[4];
        for (int r = 0; r < 3; ++r) {
            pn[r] = p[r] + dt * v[r];
            vn[r] = v[r] + dt * F[3 * j + r] / P->mass;
            wn[r] = w[r] + dt * wdot[r];
        }
        double wnorm = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (wnorm > 0.0) {
            double half = 0.5 * wnorm * dt;
            double dq[4] = {cos(half), sin(half) * w[0] / wnorm, sin(half) * w[1] / wnorm,
                            sin(half) * w[2] / wnorm};
            orc_quat_mul(q, dq, qn);
        } else {
            for (int r = 0; r < 4; ++r) qn[r] = q[r];
        }
        double qnorm = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
        for (int r = 0; r < 3; ++r) o[r] = pn[r];
        for (int r = 0; r < 4; ++r) o[3 + r] = qn[r] / qnorm;
        for (int r = 0; r < 3; ++r) o[7 + r] = vn[r];
        for (int r = 0; r < 3; ++r) o[10 + r] = wn[r];
    }
    free(F);
    free(tau);
}

/* Time derivative of one environment's state: p' = v, q' = 1/2 q (x) [0, omega] (the
 * body-frame rate multiplies on the right, as in the exponential map), v' = F/m,
 * omega' = J^-1 (tau - omega x (J omega)), the forces of orc_env_forces evaluated at x
 * with the quaternions taken at unit length (the stage states of a Runge-Kutta step
 * leave the unit sphere by O(dt^2)). dx is [N][13]. */
void orc_env_deriv(const orc_params* P, int N, const double* x, const double* rpm, int flags, const double* f_ext,
                   double* dx)
{
    double* xu = (double*)malloc(sizeof(double) * 13 * (size_t)(N > 0 ? N : 1));
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double* tau = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    memcpy(xu, x, sizeof(double) * 13 * (size_t)N);
    for (int j = 0; j < N; ++j) {
        double* q = xu + 13 * j + 3;
        const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int r = 0; r < 4; ++r) q[r] /= qn;
    }
    orc_env_forces(P, N, xu, rpm, flags, f_ext, F, tau);
    const double J[3] = {P->Jxx, P->Jyy, P->Jzz};
    for (int j = 0; j < N; ++j) {
        const double* s = x + 13 * j;
        double* d = dx + 13 * j;
        const double* q = s + 3;
        const double* w = s + 10;
        const double wq[4] = {0.0, w[0], w[1], w[2]};
        double qd[4];
        orc_quat_mul(q, wq, qd);
        for (int r = 0; r < 3; ++r) d[r] = s[7 + r];
        for (int r = 0; r < 4; ++r) d[3 + r] = 0.5 * qd[r];
        for (int r = 0; r < 3; ++r) d[7 + r] = F[3 * j + r] / P->mass;
        orc_angular_accel(J, tau + 3 * j, w, d + 10);
    }
    free(xu);
    free(F);
    free(tau);
}

/* One substep of classical fourth-order Runge-Kutta for one environment (the MuJoCo
 * modes of Table "Physics modes" integrate with RK4). Reading: the 13-d states of all
 * drones of the environment advance jointly (the downwash couples them, so every stage
 * evaluates every force at that stage's states), k1 = f(x), k2 = f(x + dt/2 k1),
 * k3 = f(x + dt/2 k2), k4 = f(x + dt k3), x+ = x + dt/6 (k1 + 2 k2 + 2 k3 + k4), the
 * quaternion advanced like the other components and renormalised at the end. */
void orc_substep_rk4(const orc_params* P, int N, const double* x_in, const double* rpm, int flags,
                     const double* f_ext, double dt, double* x_out)
{
    const size_t n13 = 13 * (size_t)(N > 0 ? N : 1);
    double* k1 = (double*)malloc(sizeof(double) * n13);
    double* k2 = (double*)malloc(sizeof(double) * n13);
    double* k3 = (double*)malloc(sizeof(double) * n13);
    double* k4 = (double*)malloc(sizeof(double) * n13);
    double* xs = (double*)malloc(sizeof(double) * n13);
    const size_t m = 13 * (size_t)N;
    orc_env_deriv(P, N, x_in, rpm, flags, f_ext, k1);
    for (size_t i = 0; i < m; ++i) xs[i] = x_in[i] + 0.5 * dt * k1[i];
    orc_env_deriv(P, N, xs, rpm, flags, f_ext, k2);
    for (size_t i = 0; i < m; ++i) xs[i] = x_in[i] + 0.5 * dt * k2[i];
    orc_env_deriv(P, N, xs, rpm, flags, f_ext, k3);
    for (size_t i = 0; i < m; ++i) xs[i] = x_in[i] + dt * k3[i];
    orc_env_deriv(P, N, xs, rpm, flags, f_ext, k4);
    for (size_t i = 0; i < m; ++i) x_out[i] = x_in[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    for (int j = 0; j < N; ++j) {
        double* q = x_out + 13 * j + 3;
        const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int r = 0; r < 4; ++r) q[r] /= qn;
    }
    free(k1);
    free(k2);
    free(k3);
    free(k4);
    free(xs);
}

/* ---- PID waypoint controller (Section 4.2.1, Table "Default PIDControl gains") ---- */

/* Solve A x = b for a 4x4 A by Gaussian elimination with partial pivoting (the
 * plain definition of the linear solve the controller performs). */
static void solve4(double A[4][4], double b[4], double x[4])
{
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < 4; ++k) {
                double t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < 4; ++r) {
            double f = A[r][c] / A[c][c];
            for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < 4; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
}

/* The allocation matrix M of Section 4.2.1: [T, tau_x, tau_y, tau_z] = M f with
 * f_i = k_f n_i^2, the rows being Eq. motor's mixing (tau_z = (k_m/k_f) sum
 * (-1)^{m_i} f_i). */
void orc_allocation_matrix(const orc_params* P, double M[16])
{
    const double r = P->km / P->kf;
    if (P->frame == ORC_FRAME_P) {
        const double L = P->arm;
        const double rows[4][4] = {{1, 1, 1, 1}, {0, L, 0, -L}, {-L, 0, L, 0}, {-r, r, -r, r}};
        for (int i = 0; i < 4; ++i)
            for (int k = 0; k < 4; ++k) M[4 * i + k] = rows[i][k];
        return;
    }
    const double l = P->arm / sqrt(2.0);
    const double rows[4][4] = {{1, 1, 1, 1}, {l, l, -l, -l}, {-l, l, l, -l}, {-r, r, -r, r}};
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k) M[4 * i + k] = rows[i][k];
}

/* Wrap an angle to [-pi, pi). */
static double wrap_pi(double a)
{
    double w = fmod(a + ORC_PI, 2.0 * ORC_PI);
    if (w < 0.0) w += 2.0 * ORC_PI;
    return w - ORC_PI;
}

/* The cascaded PID of Section 4.2.1 in its three stages. Readings, where the paper prints
 * only the structure, the gains and T = m |a*|:
 *  - position loop a* = Kp e_p + Ki I_p + Kd (v_t - v) + a_ff + g z_hat, e_p = p_t - p,
 *    with I_p = clamp(I_p + e_p dt_ctrl, +-pos_iclamp), dt_ctrl the control period, the
 *    target velocity v_t zero for waypoints and the feed-forward acceleration a_ff
 *    (DSLPIDControl's target_acc) zero unless given;
 *  - small-angle attitude target phi* = (a*_x sin psi* - a*_y cos psi*)/g,
 *    theta* = (a*_x cos psi* + a*_y sin psi*)/g;
 *  - attitude PID tau* = Kp e_eta + Ki I_eta + Kd (w_t - omega), e_eta the roll, pitch
 *    and wrapped yaw errors, I_eta clamped to +-att_iclamp, the target body rate w_t zero
 *    for waypoints;
 *  - mixer: solve M f = [T*, tau*], clip each f_i to [0, k_f MAX_RPM^2] (standing in for
 *    the unprinted torque clamp), n_i = sqrt(f_i / k_f). */
static void orc_position_loop(const orc_params* P, const double x[13], double integ[6], const double p_t[3],
                              const double v_t[3], const double a_ff[3], double psi_t, double* T, double att_t[2],
                              double ep[3])
{
    const double* p = x;
    const double* v = x + 7;
    double a[3];
    for (int r = 0; r < 3; ++r) {
        ep[r] = p_t[r] - p[r];
        double I = integ[r] + ep[r] * P->dt_ctrl;
        if (I > P->pos_iclamp) I = P->pos_iclamp;
        if (I < -P->pos_iclamp) I = -P->pos_iclamp;
        integ[r] = I;
        a[r] = P->pos_kp[r] * ep[r] + P->pos_ki[r] * I + P->pos_kd[r] * (v_t[r] - v[r]);
        a[r] += a_ff[r];
    }
    a[2] += P->g;
    *T = P->mass * sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double phi_t = (a[0] * sin(psi_t) - a[1] * cos(psi_t)) / P->g;
    double theta_t = (a[0] * cos(psi_t) + a[1] * sin(psi_t)) / P->g;
    att_t[0] = phi_t;
    att_t[1] = theta_t;
}

static void orc_attitude_loop(const orc_params* P, const double x[13], double integ[6], double phi_t,
                              double theta_t, double psi_t, const double w_t[3], double tau[3], double* yaw_err)
{
    const double* q = x + 3;
    const double* w = x + 10;
    double rpy[3];
    orc_rpy(q, rpy);
    double ee[3] = {phi_t - rpy[0], theta_t - rpy[1], wrap_pi(psi_t - rpy[2])};
    for (int r = 0; r < 3; ++r) {
        double I = integ[3 + r] + ee[r] * P->dt_ctrl;
        if (I > P->att_iclamp) I = P->att_iclamp;
        if (I < -P->att_iclamp) I = -P->att_iclamp;
        integ[3 + r] = I;
        tau[r] = P->att_kp[r] * ee[r] + P->att_ki[r] * I + P->att_kd[r] * (w_t[r] - w[r]);
    }
    if (yaw_err) *yaw_err = ee[2];
}

static void orc_mix(const orc_params* P, double T, const double tau[3], double rpm[4])
{
    double M[16], A[4][4], b[4] = {T, tau[0], tau[1], tau[2]}, f[4];
    orc_allocation_matrix(P, M);
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k) A[i][k] = M[4 * i + k];
    solve4(A, b, f);
    const double maxrpm = orc_max_rpm(P);
    const double fmax_ = P->kf * maxrpm * maxrpm;
    for (int i = 0; i < 4; ++i) {
        double fi = f[i];
        if (fi < 0.0) fi = 0.0;
        if (fi > fmax_) fi = fmax_;
        rpm[i] = sqrt(fi / P->kf);
    }
}

/* DSLPIDControl's setpoint limiter: the setpoint sp = [x, y, z, psi] moves towards the
 * waypoint by at most sp_rate_pos dt_ctrl (Euclidean distance) and sp_rate_yaw dt_ctrl
 * (wrapped yaw difference) per control step. Reading: a setpoint whose x is NaN has not
 * been set and starts at the drone's position and yaw. */
void orc_dsl_setpoint(const orc_params* P, const double x[13], const double wp[4], double sp[4])
{
    if (isnan(sp[0])) {
        double rpy[3];
        orc_rpy(x + 3, rpy);
        for (int r = 0; r < 3; ++r) sp[r] = x[r];
        sp[3] = rpy[2];
    }
    double d[3], n2 = 0.0;
    for (int r = 0; r < 3; ++r) {
        d[r] = wp[r] - sp[r];
        n2 += d[r] * d[r];
    }
    const double lim = P->sp_rate_pos * P->dt_ctrl;
    const double n = sqrt(n2);
    const double s = n > lim ? lim / n : 1.0;
    for (int r = 0; r < 3; ++r) sp[r] += s * d[r];
    double dy = wrap_pi(wp[3] - sp[3]);
    const double ly = P->sp_rate_yaw * P->dt_ctrl;
    if (dy > ly) dy = ly;
    if (dy < -ly) dy = -ly;
    sp[3] = wrap_pi(sp[3] + dy);
}

/* One call of the cascaded PID (computeControl) for one drone towards a waypoint. x is
 * the 13-d state, integ[6] = [position error integral (3), attitude error integral (3)]
 * (updated in place), wp = [x*, y*, z*, psi*], a_ff the feed-forward acceleration (NULL:
 * zero); zero target velocity and body rate. With the DSL controller and a setpoint sp
 * (updated in place), the loops track the rate-limited setpoint instead of wp.
 * Returns (rpm, pos_error, yaw_error) like computeControl. */
void orc_pid_ff(const orc_params* P, const double x[13], double integ[6], double* sp, const double wp[4],
                const double* a_ff, double rpm[4], double pos_err[3], double* yaw_err)
{
    static const double zero[3] = {0.0, 0.0, 0.0};
    const double* tgt = wp;
    if (P->controller == ORC_CTRL_DSL && sp) {
        orc_dsl_setpoint(P, x, wp, sp);
        tgt = sp;
    }
    double T, att[2], ep[3], tau[3];
    orc_position_loop(P, x, integ, tgt, zero, a_ff ? a_ff : zero, tgt[3], &T, att, ep);
    orc_attitude_loop(P, x, integ, att[0], att[1], tgt[3], zero, tau, yaw_err);
    orc_mix(P, T, tau, rpm);
    if (pos_err) {
        for (int r = 0; r < 3; ++r) pos_err[r] = ep[r];
    }
}

void orc_pid(const orc_params* P, const double x[13], double integ[6], const double wp[4],
             double rpm[4], double pos_err[3], double* yaw_err)
{
    orc_pid_ff(P, x, integ, NULL, wp, NULL, rpm, pos_err, yaw_err);
}

/* Normalized RPM action (Table "Action types"; the tasks map actions in [-1, 1] to RPMs,
 * the map itself is not printed). Reading: a clipped to [-1, 1], -1 -> 0, 0 -> HOVER_RPM,
 * 1 -> MAX_RPM, linear on each side of hover. */
double orc_normalized_rpm(const orc_params* P, double a)
{
    if (a < -1.0) a = -1.0;
    if (a > 1.0) a = 1.0;
    const double hover = orc_hover_rpm(P), maxrpm = orc_max_rpm(P);
    return a <= 0.0 ? hover * (1.0 + a) : hover + (maxrpm - hover) * a;
}

/* Action -> four RPMs for one drone (Table "Action types", converted in
 * _preprocessAction):
 *  RPM        the four speeds clipped to [0, MAX_RPM];
 *  RPM_NORM   four normalized values (orc_normalized_rpm);
 *  ONE_D_RPM  act[0] normalized, the same speed on all four motors;
 *  PID        waypoint [x, y, z, psi] (orc_pid_ff; sp the DSL setpoint or NULL);
 *  VEL        body-frame [v_x, v_y, v_z, omega_z] through the PID: reading, the position
 *             loop holds the current position (e_p = 0) with target velocity R v_body,
 *             and the attitude loop holds the current yaw with target body rate
 *             [0, 0, omega_z];
 *  ATTITUDE   [T, phi*, theta*, yaw rate]: reading, T the collective thrust in N, the
 *             attitude loop towards phi*, theta* and the current yaw with target body rate
 *             [0, 0, yaw rate], then the mixer.
 * integ is updated as the loops run. */
void orc_action_to_rpm(const orc_params* P, int type, const double x[13], double integ[6], double* sp,
                       const double act[4], double rpm[4])
{
    if (type == ORC_ACT_PID) {
        orc_pid_ff(P, x, integ, sp, act, NULL, rpm, NULL, NULL);
    } else if (type == ORC_ACT_RPM_NORM) {
        for (int i = 0; i < 4; ++i) rpm[i] = orc_normalized_rpm(P, act[i]);
    } else if (type == ORC_ACT_ONE_D_RPM) {
        const double r = orc_normalized_rpm(P, act[0]);
        for (int i = 0; i < 4; ++i) rpm[i] = r;
    } else if (type == ORC_ACT_VEL || type == ORC_ACT_ATTITUDE) {
        double rpy[3], tau[3], T, att[2], ep[3];
        orc_rpy(x + 3, rpy);
        const double w_t[3] = {0.0, 0.0, act[3]};
        if (type == ORC_ACT_VEL) {
            double R[9], v_t[3];
            orc_rotation(x + 3, R);
            for (int r = 0; r < 3; ++r) v_t[r] = R[3 * r] * act[0] + R[3 * r + 1] * act[1] + R[3 * r + 2] * act[2];
            static const double no_ff[3] = {0.0, 0.0, 0.0};
            orc_position_loop(P, x, integ, x, v_t, no_ff, rpy[2], &T, att, ep);
        } else {
            T = act[0];
            att[0] = act[1];
            att[1] = act[2];
        }
        orc_attitude_loop(P, x, integ, att[0], att[1], rpy[2], w_t, tau, NULL);
        orc_mix(P, T, tau, rpm);
    } else {
        const double maxrpm = orc_max_rpm(P);
        for (int i = 0; i < 4; ++i) {
            double r = act[i];
            if (r < 0.0) r = 0.0;
            if (r > maxrpm) r = maxrpm;
            rpm[i] = r;
        }
    }
}

/* ---- observations (Section 3.4.4) ---- */

/* KIN observation: [p(3), q(4), rpy(3), v(3), omega(3), a_{t-1}(4)] (20 values).
 * a_{t-1} is read as the four RPMs applied over the last control step. */
void orc_kin(const double x[13], const double a_prev[4], double out[20])
{
    double rpy[3];
    orc_rpy(x + 3, rpy);
    for (int r = 0; r < 3; ++r) out[r] = x[r];
    for (int r = 0; r < 4; ++r) out[3 + r] = x[3 + r];
    for (int r = 0; r < 3; ++r) out[7 + r] = rpy[r];
    for (int r = 0; r < 3; ++r) out[10 + r] = x[7 + r];
    for (int r = 0; r < 3; ++r) out[13 + r] = x[10 + r];
    for (int r = 0; r < 4; ++r) out[16 + r] = a_prev[r];
}

/* Neighbourhood-adjacency observation (the abstract's "neighbourhood adjacency
 * information"; the format is not printed). Reading: the 4 nearest other drones
 * of the same environment by Euclidean distance, ties to the lower index, padded
 * with index -1 and zero features when the environment has fewer than 5 drones;
 * features per neighbour i of drone j: [p_i - p_j, v_i - v_j]. Distances, the
 * selection and the features are all taken in double precision. A drone whose
 * squared distance is not finite (a NaN or infinite position) is not listed.
 * idx_base is added to the local indices written. */
void orc_knn(int N, const double* x, int j, int idx_base, int32_t idx[4], double rel[24])
{
    double bestd[4];
    int besti[4];
    int nb = 0;
    for (int i = 0; i < N; ++i) {
        if (i == j) continue;
        double d2 = 0.0;
        for (int r = 0; r < 3; ++r) {
            const double d = x[13 * i + r] - x[13 * j + r];
            d2 += d * d;
        }
        if (!isfinite(d2)) continue;
        /* insert (d2, i) into the sorted list; strict '<' keeps the lower index first */
        int pos = nb;
        while (pos > 0 && d2 < bestd[pos - 1]) --pos;
        if (pos >= 4) continue;
        int last = nb < 4 ? nb : 3;
        for (int k = last; k > pos; --k) {
            bestd[k] = bestd[k - 1];
            besti[k] = besti[k - 1];
        }
        bestd[pos] = d2;
        besti[pos] = i;
        if (nb < 4) ++nb;
    }
    for (int k = 0; k < 4; ++k) {
        if (k < nb) {
            int i = besti[k];
            idx[k] = idx_base + i;
            for (int r = 0; r < 3; ++r) {
                rel[6 * k + r] = x[13 * i + r] - x[13 * j + r];
                rel[6 * k + 3 + r] = x[13 * i + 7 + r] - x[13 * j + 7 + r];
            }
        } else {
            idx[k] = -1;
            for (int r = 0; r < 6; ++r) rel[6 * k + r] = 0.0;
        }
    }
}

/* ---- batched driver: K control steps over a CSR batch of environments ---- */

/* ---- domain randomization and wind ---- */

/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014): the output function of its counter-based form. Called with the state
 * before its increment by the golden gamma, so orc_splitmix64(k * gamma) is the (k+1)-th
 * output of the generator started from state 0 (pinned against the published sequence). */
uint64_t orc_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* U[0, 1) with 24 random bits (exact in float and double) for the counters (seed, stream,
 * step, index, comp): each field is mixed in by one SplitMix64 round. */
double orc_uniform(uint64_t seed, uint64_t stream, uint64_t step, uint64_t index, uint64_t comp)
{
    uint64_t h = orc_splitmix64(seed);
    h = orc_splitmix64(h ^ stream);
    h = orc_splitmix64(h ^ step);
    h = orc_splitmix64(h ^ index);
    h = orc_splitmix64(h ^ comp);
    return (double)(h >> 40) * (1.0 / 16777216.0);
}

/* The physics model of one environment under its domain-randomization row: the factors
 * scale mass, inertia, arm, k_f, k_m, c_xy, c_z, C_gnd, C1 and g (h_clip, a numerical
 * guard, stays nominal). */
void orc_params_randomized(const orc_params* P, const double* dr, orc_params* Pe)
{
    *Pe = *P;
    Pe->mass *= dr[ORC_DR_MASS];
    Pe->Jxx *= dr[ORC_DR_J + 0];
    Pe->Jyy *= dr[ORC_DR_J + 1];
    Pe->Jzz *= dr[ORC_DR_J + 2];
    Pe->arm *= dr[ORC_DR_ARM];
    Pe->kf *= dr[ORC_DR_KF];
    Pe->km *= dr[ORC_DR_KM];
    Pe->c_xy *= dr[ORC_DR_CXY];
    Pe->c_z *= dr[ORC_DR_CZ];
    Pe->c_gnd *= dr[ORC_DR_CGND];
    Pe->dw_c1 *= dr[ORC_DR_C1];
    Pe->g *= dr[ORC_DR_G];
}

/* One control step of an environment's WindField (Section 3.5): advances the wind state
 * ws[ORC_WIND_STATE] of environment `env` and returns the direct force F_dir [N] (gusts,
 * sinusoid) and the wind velocity v_w [m/s] the quadratic drag sees (steady wind plus
 * Dryden turbulence). Readings where the paper gives the models only in outline:
 *  CONSTANT   v_w += the steady wind; drag on drone j: k |v_rel| v_rel, v_rel = v_w - v_j
 *             (= 1/2 rho C_d A |v_rel|^2 v_rel_hat), also with DRYDEN alone;
 *  DRYDEN     per component x <- alpha x + sigma sqrt(1 - alpha^2) xi, xi ~ N(0, 1) (Box-Muller
 *             on the counter-based uniforms), alpha = exp(-dt_ctrl V / L),
 *             L = h / (0.177 + 8.23e-4 h)^1.2 with the environment's reference altitude h,
 *             the same L for all three components; v_w += x;
 *  GUST       an idle field starts a gust with the given probability per control step, in a
 *             direction uniform on the sphere; the gust force is A sin(pi s) d for its phase
 *             s = 0, dt_ctrl/T, ... while s <= 1;
 *  SINUSOIDAL F += A [sin wt, cos wt, 0.3 sin 2wt], t = steps dt_ctrl;
 *  COMBINED   every bit set. */
void orc_wind_step(const orc_params* P, const double* dr, double* ws, uint64_t seed, int64_t env, double F_dir[3],
                   double v_w[3])
{
    const int model = (int)dr[ORC_DR_WIND];
    const double dt = P->dt_ctrl;
    const uint64_t step = (uint64_t)ws[7];
    for (int r = 0; r < 3; ++r) F_dir[r] = v_w[r] = 0.0;
    if (model & ORC_WIND_CONSTANT)
        for (int r = 0; r < 3; ++r) v_w[r] += dr[ORC_DR_VWIND + r];
    if (model & ORC_WIND_DRYDEN) {
        const double h = dr[ORC_DR_DRY_H];
        const double L = h / pow(0.177 + 8.23e-4 * h, 1.2);
        const double alpha = exp(-dt * dr[ORC_DR_DRY_V] / L);
        const double u1 = 1.0 - orc_uniform(seed, ORC_STREAM_WIND, step, (uint64_t)env, 0);
        const double u2 = orc_uniform(seed, ORC_STREAM_WIND, step, (uint64_t)env, 1);
        const double u3 = 1.0 - orc_uniform(seed, ORC_STREAM_WIND, step, (uint64_t)env, 2);
        const double u4 = orc_uniform(seed, ORC_STREAM_WIND, step, (uint64_t)env, 3);
        const double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
        const double xi[3] = {r1 * cos(2.0 * ORC_PI * u2), r1 * sin(2.0 * ORC_PI * u2), r2 * cos(2.0 * ORC_PI * u4)};
        for (int r = 0; r < 3; ++r) {
            ws[r] = alpha * ws[r] + dr[ORC_DR_DRY_SIGMA] * sqrt(1.0 - alpha * alpha) * xi[r];
            v_w[r] += ws[r];
        }
    }
    if (model & ORC_WIND_GUST) {
        if (ws[3] < 0.0) {
            const double u = orc_uniform(seed, ORC_STREAM_WIND, step, (uint64_t)env, 4);
            if (u < dr[ORC_DR_GUST_P]) {
                const double z = 2.0 * orc_uniform(seed, ORC_STREAM_WIND, step, (uint64_t)env, 5) - 1.0;
                const double ph = 2.0 * ORC_PI * orc_uniform(seed, ORC_STREAM_WIND, step, (uint64_t)env, 6);
                const double rho = sqrt(1.0 - z * z);
                ws[3] = 0.0;
                ws[4] = rho * cos(ph);
                ws[5] = rho * sin(ph);
                ws[6] = z;
            }
        }
        if (ws[3] >= 0.0) {
            const double a = dr[ORC_DR_GUST_A] * sin(ORC_PI * ws[3]);
            for (int r = 0; r < 3; ++r) F_dir[r] += a * ws[4 + r];
            const double s_next = ws[3] + dt / dr[ORC_DR_GUST_T];
            ws[3] = s_next > 1.0 ? -1.0 : s_next;
        }
    }
    if (model & ORC_WIND_SINUSOIDAL) {
        const double t = (double)step * dt, w = dr[ORC_DR_SIN_W], A = dr[ORC_DR_SIN_A];
        F_dir[0] += A * sin(w * t);
        F_dir[1] += A * cos(w * t);
        F_dir[2] += A * 0.3 * sin(2.0 * w * t);
    }
    ws[7] = (double)(step + 1);
}

/* ---- episode reset under domain randomization (Section 3.5) ---- */

/* The initial state of one drone for one episode, the "init" row of Table "Recommended
 * domain-randomization ranges" (p0 +-0.2 m, RPY0 +-0.1 rad, v0 +-0.5 m/s, drawn at every
 * reset like the rest of the table): each component is its nominal value plus a uniform
 * draw in [-r, r],
 *   p0   = nominal[0..2] + r[0] (2 u_k - 1), k = 0, 1, 2
 *   RPY0 = (0, 0, nominal[3]) + r[1] (2 u_k - 1), k = 3, 4, 5 (roll, pitch, yaw)
 *   v0   = r[2] (2 u_k - 1), k = 6, 7, 8
 * with u_k = orc_uniform(seed, ORC_STREAM_INIT, episode, drone, k); the attitude is the
 * quaternion of R = Rz(yaw) Ry(pitch) Rx(roll) (the ZYX convention orc_rpy inverts), the body
 * rate zero. x = [p, q, v, omega]. */
void orc_reset_state(const double nominal[4], const double r[3], uint64_t seed, uint64_t episode, uint64_t drone,
                     double x[13])
{
    double u[9];
    for (int k = 0; k < 9; ++k) u[k] = 2.0 * orc_uniform(seed, ORC_STREAM_INIT, episode, drone, (uint64_t)k) - 1.0;
    const double roll = r[1] * u[3], pitch = r[1] * u[4], yaw = nominal[3] + r[1] * u[5];
    const double qx[4] = {cos(0.5 * roll), sin(0.5 * roll), 0.0, 0.0};
    const double qy[4] = {cos(0.5 * pitch), 0.0, sin(0.5 * pitch), 0.0};
    const double qz[4] = {cos(0.5 * yaw), 0.0, 0.0, sin(0.5 * yaw)};
    double qzy[4];
    orc_quat_mul(qz, qy, qzy);
    for (int k = 0; k < 3; ++k) x[k] = nominal[k] + r[0] * u[k];
    orc_quat_mul(qzy, qx, x + 3);
    for (int k = 0; k < 3; ++k) x[7 + k] = r[2] * u[6 + k];
    for (int k = 0; k < 3; ++k) x[10 + k] = 0.0;
}

/* The sticky per-episode observation bias of recommendation (iii) of Section 3.5 ("coupling
 * DR with a sticky per-episode bias on the observation"; its size is not printed): one
 * Gaussian offset per KIN channel that the sensor noise also perturbs, drawn at the reset
 * and held for the episode, b_k = sigma[k / 3] xi_k for the channels k = 0..11 (position
 * 0-2, roll/pitch/yaw 3-5, velocity 6-8, body rate 9-11), xi by Box-Muller on the pairs of
 * uniforms (seed, ORC_STREAM_BIAS, episode, drone, 2m) and (.., 2m + 1): xi_2m = rho cos(2 pi
 * u_2m+1), xi_2m+1 = rho sin(2 pi u_2m+1), rho = sqrt(-2 ln(1 - u_2m)). */
void orc_obs_bias(const double sigma[4], uint64_t seed, uint64_t episode, uint64_t drone, double b[12])
{
    for (int m = 0; m < 6; ++m) {
        const double u1 = 1.0 - orc_uniform(seed, ORC_STREAM_BIAS, episode, drone, (uint64_t)(2 * m));
        const double u2 = orc_uniform(seed, ORC_STREAM_BIAS, episode, drone, (uint64_t)(2 * m + 1));
        const double rho = sqrt(-2.0 * log(u1));
        b[2 * m] = sigma[(2 * m) / 3] * rho * cos(2.0 * ORC_PI * u2);
        b[2 * m + 1] = sigma[(2 * m + 1) / 3] * rho * sin(2.0 * ORC_PI * u2);
    }
}

/* Runs K control steps (Section 3.4.2: sim_freq/ctrl_freq substeps per step) for
 * n_envs environments laid out in CSR order (drones of env e are
 * env_off[e] .. env_off[e+1]-1). Per control step and environment: the action of
 * each drone becomes four RPMs by the environment's action type (orc_action_to_rpm),
 * the RPMs are held over n_sub substeps of dt_sim, and a_prev records them. After the
 * last step the observations are written when kin is not NULL.
 *   x        [n][13]   state, updated in place
 *   integ    [n][6]    PID integrals, updated in place
 *   a_prev   [n][4]    last applied RPMs, written
 *   actions  [K][n][4] one action per drone (RPMs, waypoints, velocities, ...)
 *   kin      [n][20], nbr_idx [n][4], nbr_rel [n][24] (optional)
 *   setpoint [n][4]    DSL setpoints, updated in place (required with the DSL
 *                      controller, else ignored; may be NULL)
 *   dr                 domain randomization and wind (NULL: none):
 *     env_dr [n_envs][ORC_DR_PARAMS]; motor [n][4] rotor speeds (the lag's state, NaN =
 *     not set: starts at the first command); hist [depth][n][4] actions received (the
 *     latency's shift register, NaN = empty: filled with the first action); wind
 *     [n_envs][ORC_WIND_STATE]; seed of the wind draws.
 *   Per control step and drone, with dr: the action received enters the shift register
 *   and the one received `delay` steps ago is applied; it becomes RPMs through the
 *   nominal controller (recorded in a_prev); each motor's command is its RPM times its
 *   bias, saturated at MAX_RPM times the factor; the wind force (orc_wind_step, drag from
 *   the drone's velocity at the step's start) is held over the substeps; before each
 *   substep every rotor speed relaxes towards its command, n <- c + (n - c) exp(-dt/tau)
 *   (exact for a first-order lag under a constant command; tau = 0: n = c), and the
 *   substep integrates the environment's randomized model with these speeds.
 *   Observations under dr (the sensor group of the randomization table): with a sensor
 *   delay of one control step the KIN observation reports the state and the RPMs of the
 *   last step's start; KIN positions, roll/pitch/yaw, velocities and body rates get
 *   Gaussian noise of the row's sigmas, drawn from the counters (seed, ORC_STREAM_OBS, the
 *   environment's wind step of the last step, drone, component 0..11; Box-Muller on the
 *   pairs (0, 1), ..., (10, 11): position 0-2, rpy 3-5, velocity 6-8, body rate 9-11); the
 *   neighbour observation is not delayed and carries no noise. obs_bias [n][12] (or NULL),
 *   the sticky per-episode bias of orc_obs_bias, is added to the same KIN channels as the
 *   noise (position, roll/pitch/yaw, velocity, body rate), delayed or not.
 * Returns 0, or -1 on a bad argument. */
typedef struct {
    const double* env_dr;
    double* motor;
    double* hist;
    int32_t depth;
    double* wind;
    uint64_t seed;
    const double* obs_bias;
} orc_dr;

int orc_control_steps(const orc_params* P, int n_envs, const int32_t* env_off, const int32_t* env_flags,
                      const int32_t* env_act, double* x, double* integ, double* a_prev, const double* actions,
                      int K, int n_sub, double* kin, int32_t* nbr_idx, double* nbr_rel, double* setpoint,
                      const orc_dr* dr)
{
    if (n_envs < 0 || K < 0 || n_sub < 1) return -1;
    if (P->controller == ORC_CTRL_DSL && !setpoint) return -1;
    if (dr && (!dr->env_dr || !dr->motor || !dr->hist || dr->depth < 1 || !dr->wind)) return -1;
    int maxN = 0;
    for (int e = 0; e < n_envs; ++e) {
        int N = env_off[e + 1] - env_off[e];
        if (N < 0) return -1;
        if (N > maxN) maxN = N;
    }
    const int64_t n = n_envs > 0 ? env_off[n_envs] : 0;
    if (dr) {
        for (int e = 0; e < n_envs; ++e) {
            const double d = dr->env_dr[(size_t)e * ORC_DR_PARAMS + ORC_DR_DELAY];
            if (!(d >= 0.0) || d != floor(d) || d >= dr->depth) return -1;
            const double od = dr->env_dr[(size_t)e * ORC_DR_PARAMS + ORC_DR_OBS_DELAY];
            if (od != 0.0 && od != 1.0) return -1;
        }
    }
    /* the state and RPMs at the last step's start, for delayed observations */
    double* x_last = (dr && kin) ? (double*)malloc(sizeof(double) * 13 * (size_t)(n > 0 ? n : 1)) : NULL;
    double* a_last = (dr && kin) ? (double*)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1)) : NULL;
    const size_t nb = (size_t)(maxN > 0 ? maxN : 1);
    double* rpm = (double*)malloc(sizeof(double) * 4 * nb);
    double* cmd = (double*)malloc(sizeof(double) * 4 * nb);
    double* fext = (double*)malloc(sizeof(double) * 3 * nb);
    double* tmp = (double*)malloc(sizeof(double) * 13 * nb);
    const double maxrpm = orc_max_rpm(P);
    for (int k = 0; k < K; ++k) {
        const double* act = actions + (size_t)k * (size_t)n * 4;
        if (x_last && k == K - 1) {
            memcpy(x_last, x, sizeof(double) * 13 * (size_t)n);
            memcpy(a_last, a_prev, sizeof(double) * 4 * (size_t)n);
        }
        for (int e = 0; e < n_envs; ++e) {
            const int b = env_off[e], N = env_off[e + 1] - env_off[e];
            const double* row = dr ? dr->env_dr + (size_t)e * ORC_DR_PARAMS : NULL;
            orc_params Pe = *P;
            double F_dir[3] = {0.0, 0.0, 0.0}, v_w[3] = {0.0, 0.0, 0.0};
            if (row) {
                orc_params_randomized(P, row, &Pe);
                orc_wind_step(P, row, dr->wind + (size_t)e * ORC_WIND_STATE, dr->seed, e, F_dir, v_w);
            }
            const int drag_wind = row && ((int)row[ORC_DR_WIND] & (ORC_WIND_CONSTANT | ORC_WIND_DRYDEN));
            for (int j = 0; j < N; ++j) {
                const size_t g = (size_t)(b + j);
                const double* a = act + 4 * g;
                if (row) {
                    /* action latency: shift register of the actions received */
                    double* h0 = dr->hist + 4 * g;
                    const size_t hs = 4 * (size_t)n;
                    if (isnan(h0[0])) {
                        for (int d = 0; d < dr->depth; ++d)
                            for (int i = 0; i < 4; ++i) h0[d * hs + i] = a[i];
                    } else {
                        for (int d = dr->depth - 1; d > 0; --d)
                            for (int i = 0; i < 4; ++i) h0[d * hs + i] = h0[(d - 1) * hs + i];
                        for (int i = 0; i < 4; ++i) h0[i] = a[i];
                    }
                    a = h0 + (size_t)row[ORC_DR_DELAY] * hs;
                }
                orc_action_to_rpm(P, env_act[e], x + 13 * g, integ + 6 * g, setpoint ? setpoint + 4 * g : NULL, a,
                                  rpm + 4 * j);
                for (int i = 0; i < 4; ++i) a_prev[4 * g + i] = rpm[4 * j + i];
                for (int i = 0; i < 4; ++i) {
                    double c = rpm[4 * j + i];
                    if (row) {
                        c *= row[ORC_DR_BIAS + i];
                        const double sat = maxrpm * row[ORC_DR_MAXRPM];
                        if (c > sat) c = sat;
                        if (isnan(dr->motor[4 * g + i])) dr->motor[4 * g + i] = c;
                    }
                    cmd[4 * j + i] = c;
                }
                for (int r = 0; r < 3; ++r) {
                    double f = F_dir[r];
                    if (drag_wind) {
                        const double* v = x + 13 * g + 7;
                        const double vr[3] = {v_w[0] - v[0], v_w[1] - v[1], v_w[2] - v[2]};
                        const double m = sqrt(vr[0] * vr[0] + vr[1] * vr[1] + vr[2] * vr[2]);
                        f += row[ORC_DR_KDRAG] * m * vr[r];
                    }
                    fext[3 * j + r] = f;
                }
            }
            const double lag = row && row[ORC_DR_TAU] > 0.0 ? exp(-P->dt_sim / row[ORC_DR_TAU]) : 0.0;
            for (int s = 0; s < n_sub; ++s) {
                const double* speeds = cmd;
                if (row) {
                    for (int j = 0; j < N; ++j)
                        for (int i = 0; i < 4; ++i) {
                            double* m = dr->motor + 4 * (size_t)(b + j) + i;
                            const double c = cmd[4 * j + i];
                            *m = c + (*m - c) * lag;
                            rpm[4 * j + i] = *m;
                        }
                    speeds = rpm;
                }
                if (P->integrator == ORC_RK4)
                    orc_substep_rk4(&Pe, N, x + 13 * (size_t)b, speeds, env_flags[e], row ? fext : NULL, P->dt_sim,
                                    tmp);
                else
                    orc_substep(&Pe, N, x + 13 * (size_t)b, speeds, env_flags[e], row ? fext : NULL, P->dt_sim, tmp);
                memcpy(x + 13 * (size_t)b, tmp, sizeof(double) * 13 * (size_t)N);
            }
        }
    }
    if (kin) {
        for (int e = 0; e < n_envs; ++e) {
            const int b = env_off[e], N = env_off[e + 1] - env_off[e];
            const double* row = dr ? dr->env_dr + (size_t)e * ORC_DR_PARAMS : NULL;
            const int delayed = row && x_last && K > 0 && row[ORC_DR_OBS_DELAY] == 1.0;
            for (int j = 0; j < N; ++j) {
                const size_t g = (size_t)(b + j);
                double* o = kin + 20 * g;
                if (delayed) orc_kin(x_last + 13 * g, a_last + 4 * g, o);
                else orc_kin(x + 13 * g, a_prev + 4 * g, o);
                if (row && K > 0) {
                    /* Gaussian sensor noise (Box-Muller on counter-based uniforms) */
                    const uint64_t step = (uint64_t)dr->wind[(size_t)e * ORC_WIND_STATE + 7] - 1;
                    double xi[12];
                    for (int m = 0; m < 6; ++m) {
                        const double u1 = 1.0 - orc_uniform(dr->seed, ORC_STREAM_OBS, step, g, 2 * m);
                        const double u2 = orc_uniform(dr->seed, ORC_STREAM_OBS, step, g, 2 * m + 1);
                        const double r = sqrt(-2.0 * log(u1));
                        xi[2 * m] = r * cos(2.0 * ORC_PI * u2);
                        xi[2 * m + 1] = r * sin(2.0 * ORC_PI * u2);
                    }
                    for (int r = 0; r < 3; ++r) {
                        o[r] += row[ORC_DR_NOISE_P] * xi[r];           /* KIN 0-2: position */
                        o[7 + r] += row[ORC_DR_NOISE_RPY] * xi[3 + r]; /* KIN 7-9: roll, pitch, yaw */
                        o[10 + r] += row[ORC_DR_NOISE_V] * xi[6 + r];  /* KIN 10-12: velocity */
                        o[13 + r] += row[ORC_DR_NOISE_W] * xi[9 + r];  /* KIN 13-15: body rate */
                    }
                    if (dr->obs_bias) {
                        const double* bb = dr->obs_bias + 12 * g;
                        for (int r = 0; r < 3; ++r) {
                            o[r] += bb[r];
                            o[7 + r] += bb[3 + r];
                            o[10 + r] += bb[6 + r];
                            o[13 + r] += bb[9 + r];
                        }
                    }
                }
                if (nbr_idx && nbr_rel)
                    orc_knn(N, x + 13 * (size_t)b, j, b, nbr_idx + 4 * (size_t)(b + j),
                            nbr_rel + 24 * (size_t)(b + j));
            }
        }
    }
    free(rpm);
    free(cmd);
    free(fext);
    free(tmp);
    free(x_last);
    free(a_last);
    return 0;
}
