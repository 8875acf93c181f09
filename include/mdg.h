/*
 * mdg.h — C ABI of the GB300-native batched multi-drone dynamics library.
 *
 * The library advances many independent environments of Crazyflie 2.x quadrotors
 * with the explicit dynamics of MuJoCo-Drones-Gym (arxiv 2606.08039): the motor
 * model (Eq. motor), ground effect (Eq. ground), blade drag (Eq. drag) and
 * inter-drone downwash (Eq. downwash) of Section 3.1, explicit Euler integration
 * with the closed-form quaternion exponential map (Section 3.2, DYN mode), the
 * cascaded PID waypoint controller (Section 4.2.1, Table "Default PIDControl
 * gains") and the KIN / neighbour observations (Section 3.4.4 and the abstract).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: MDG_OK (0) or a negative MDG_ERR_* code. Argument errors are
 *    found on the host before anything is launched; mdg_last_error() then holds a
 *    message (thread-local, valid until the next call on that thread).
 *  - Device pointers are plain CUDA device addresses owned by the caller (for
 *    instance torch tensors); the library never frees them. Each must be 16-byte
 *    aligned and hold the documented number of elements.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Every compute call is asynchronous on that stream.
 *  - Drones are numbered in CSR order: the drones of environment e are
 *    env_off[e] .. env_off[e+1]-1, env_off being the prefix sum of drones_per_env.
 *  - A handle is bound to the CUDA device current when it was created; it is not
 *    thread-safe (one host thread at a time).
 *
 * State layout (device, float32, caller-owned): MDG_STATE_PLANES planes of
 * n_drones float4 each, plane k of drone i at float offset 4*(k*n_drones + i):
 *   plane 0: p.x  p.y  p.z  q.w        (world position [m]; body-to-world quaternion)
 *   plane 1: q.x  q.y  q.z  v.x        (world velocity [m/s])
 *   plane 2: v.y  v.z  w.x  w.y        (body-frame angular velocity [rad/s])
 *   plane 3: w.z  Ip.x Ip.y Ip.z       (PID position-error integral [m s])
 *   plane 4: Ia.r Ia.p Ia.y  -         (PID attitude-error integral [rad s])
 *   plane 5: a0   a1   a2   a3         (RPMs applied during the last control step)
 * The quaternion is [w, x, y, z] (MuJoCo's order, Section 3.1.1); callers keep it
 * unit-norm and the library renormalises it after every substep.
 */
#ifndef MDG_H
#define MDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MDG_OK 0
#define MDG_ERR_ARG (-1)         /* invalid argument (message in mdg_last_error) */
#define MDG_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define MDG_ERR_NONFINITE (-3)   /* reported through mdg_status: a state became non-finite */
#define MDG_ERR_UNSUPPORTED (-4) /* a valid request this build does not implement */
#define MDG_ERR_TIMEOUT (-5)     /* mdg_sync: the stream was still busy when its limit ran out */

/* Physics-mode bits per environment (Table "Physics modes"): any subset of the
 * three aerodynamic effects on top of the explicit integrator. */
#define MDG_GND 1u  /* ground effect, Eq. ground */
#define MDG_DRAG 2u /* blade drag, Eq. drag */
#define MDG_DW 4u   /* inter-drone downwash, Eq. downwash */

/* Action types (Table "Action types"); every action is four floats per drone. */
#define MDG_ACT_RPM 0   /* action = four motor speeds [RPM], clipped to [0, MAX_RPM] */
#define MDG_ACT_PID 1   /* action = waypoint [x, y, z, yaw] for the PID controller */
#define MDG_ACT_MIXED 2 /* per-environment type, set by mdg_set_action_types */
/* Normalized speeds: four values in [-1, 1] (clipped), mapped piecewise linearly with
 * -1 -> 0, 0 -> HOVER_RPM, 1 -> MAX_RPM (the tasks' normalized actions; the map is not
 * printed, this is the library's reading). */
#define MDG_ACT_RPM_NORM 3
/* ONE_D_RPM: the first value, normalized as above, on all four motors (others ignored). */
#define MDG_ACT_ONE_D_RPM 4
/* VEL: body-frame [v_x, v_y, v_z, omega_z] through the PID: the position loop holds the
 * current position with target velocity R v_body, the attitude loop the current yaw with
 * target body rate [0, 0, omega_z]. Updates the integrals like PID. */
#define MDG_ACT_VEL 5
/* ATTITUDE: [T (N), roll*, pitch* (rad), yaw rate (rad/s)] through the attitude loop (current
 * yaw, target body rate [0, 0, yaw rate]) and the mixer. Updates the attitude integrals. */
#define MDG_ACT_ATTITUDE 6

/* Status bits written by the kernels (read with mdg_status). */
#define MDG_STATUS_NONFINITE 1u /* a drone's state became NaN or infinite */
#define MDG_STATUS_TIMEOUT 2u   /* a tensor-core kernel gave up waiting for its MMAs (bounded wait) */
#define MDG_STATUS_BOUNDS 4u    /* library built with MDG_DEBUG: a kernel found a tile, environment or
                                   list index outside its table and skipped the access */

#define MDG_STATE_PLANES 6
#define MDG_KIN_DIM 20     /* [p(3), q(4), roll/pitch/yaw(3), v(3), w(3), a_prev(4)] */
#define MDG_NBR_K 4        /* neighbours per drone */
#define MDG_NBR_FEAT 6     /* [p_i - p_j (3), v_i - v_j (3)] per neighbour */
#define MDG_MAX_ENV_DRONES 1024

typedef struct mdg_ctx* mdg_handle;

/* Model constants, SI units, double precision on the host (the kernels use float32
 * copies). Table "Drone model parameters" gives mass..prop_radius for CF2X; n is in
 * RPM, so kf [N/RPM^2] and km [N m/RPM^2] are per RPM squared. g, c_gnd, h_clip,
 * c_xy and c_z are not printed in the paper (mdg_constants_cf2x documents the
 * defaults). dw_c1..dw_c3 are Eq. downwash's (C1, C2, C3); dw_max_xy its 10 m lateral
 * cut-off; dw_dz_min an optional minimum height difference (0 = as printed). The PID
 * gains follow Table "Default PIDControl gains". dt_sim = 1/f_sim is the substep,
 * dt_ctrl = 1/f_ctrl the control period (the PID's integration step). frame selects the
 * rotor layout of Eq. motor: MDG_FRAME_X (CF2X, RACE) or MDG_FRAME_P (CF2P, the X layout
 * turned by 45 degrees: tau_x = L (F1 - F3), tau_y = L (F2 - F0)). integrator selects the
 * substep: MDG_INTEGRATOR_EULER (the DYN mode's explicit Euler with the exponential map)
 * or MDG_INTEGRATOR_RK4 (classical fourth-order Runge-Kutta on each environment's drones
 * jointly, every stage evaluating every force at that stage's states, the quaternion
 * renormalised after the substep; Table "Physics modes" lists RK4 for the MuJoCo modes).
 * gnd_heights selects where Eq. ground takes h: MDG_GND_COM (the centre of mass for all
 * four rotors, as printed) or MDG_GND_ROTOR (rotor i adds C_gnd k_f n_i^2 (r_p/(4 h_i))^2
 * with h_i = max(p_z + (R r_i)_z, h_clip), r_i its body position: L/sqrt2 (+,+), (-,+),
 * (-,-), (+,-) for X, L (+x, +y, -x, -y) for +, as the torque equations of Section 3.1.2
 * place them). */
#define MDG_FRAME_X 0
#define MDG_FRAME_P 1
#define MDG_INTEGRATOR_EULER 0
#define MDG_INTEGRATOR_RK4 1
#define MDG_GND_COM 0
#define MDG_GND_ROTOR 1
/* controller selects the cascaded PID of Section 4.2.1: MDG_CTRL_PID (PIDControl) or
 * MDG_CTRL_DSL (DSLPIDControl: its gains and halved clamps are set by
 * mdg_controller_dsl; the waypoint is tracked through a setpoint that moves towards it by
 * at most sp_rate_pos [m/s] and sp_rate_yaw [rad/s] per control period; the setpoints live
 * in a caller-owned buffer attached with mdg_set_setpoints). */
#define MDG_CTRL_PID 0
#define MDG_CTRL_DSL 1

/* Domain randomization and wind (Section 3.5: the recommended-ranges table, reset per
 * episode; "Wind and turbulence"): one row of MDG_DR_PARAMS floats per environment.
 * Factors scale the model the physics integrates (the controller keeps the nominal
 * constants: it does not know the draw). */
#define MDG_DR_PARAMS 40
#define MDG_DR_MASS 0       /* x m */
#define MDG_DR_J 1          /* x Jxx, Jyy, Jzz (1..3) */
#define MDG_DR_ARM 4        /* x L */
#define MDG_DR_KF 5         /* x k_f */
#define MDG_DR_KM 6         /* x k_m */
#define MDG_DR_CXY 7        /* x c_xy */
#define MDG_DR_CZ 8         /* x c_z */
#define MDG_DR_CGND 9       /* x C_gnd */
#define MDG_DR_C1 10        /* x downwash C1 */
#define MDG_DR_MAXRPM 11    /* x MAX_RPM: the motors saturate there */
#define MDG_DR_BIAS 12      /* per-motor speed bias (12..15): command = RPM x bias */
#define MDG_DR_G 16         /* x g */
#define MDG_DR_TAU 17       /* motor lag time constant [s] (0: none) */
#define MDG_DR_DELAY 18     /* action latency [control steps], a whole number < the history depth */
#define MDG_DR_WIND 19      /* wind model bits (MDG_WIND_*) */
#define MDG_DR_VWIND 20     /* steady wind velocity [m/s], world frame (20..22) */
#define MDG_DR_KDRAG 23     /* 1/2 rho C_d A [kg/m]: drag k |v_rel| v_rel, v_rel = wind - drone */
#define MDG_DR_GUST_P 24    /* gust trigger probability per control step */
#define MDG_DR_GUST_A 25    /* gust amplitude [N] */
#define MDG_DR_GUST_T 26    /* gust duration [s] */
#define MDG_DR_DRY_SIGMA 27 /* Dryden turbulence intensity [m/s] */
#define MDG_DR_DRY_V 28     /* Dryden airspeed V [m/s] */
#define MDG_DR_SIN_A 29     /* sinusoidal force amplitude [N] */
#define MDG_DR_SIN_W 30     /* sinusoidal angular frequency [rad/s] */
#define MDG_DR_DRY_H 31     /* Dryden reference altitude h [m] */
#define MDG_DR_NOISE_P 32   /* observation noise sigma of the KIN position [m] */
#define MDG_DR_NOISE_V 33   /* ... of the KIN velocity [m/s] */
#define MDG_DR_NOISE_RPY 34 /* ... of the KIN roll, pitch, yaw [rad] */
#define MDG_DR_NOISE_W 35   /* ... of the KIN body rate [rad/s] */
#define MDG_DR_OBS_DELAY 36 /* sensor latency [control steps]: 0 or 1 (37..39 unused) */
#define MDG_WIND_CONSTANT 1
#define MDG_WIND_GUST 2
#define MDG_WIND_DRYDEN 4
#define MDG_WIND_SINUSOIDAL 8
#define MDG_WIND_COMBINED 15
#define MDG_WIND_STATE 8    /* floats per environment: Dryden x (3), gust phase (-1 idle), gust direction (3), steps */
#define MDG_MAX_HIST_DEPTH 16
typedef struct mdg_constants {
    double mass, arm, thrust2weight, Jxx, Jyy, Jzz, kf, km, prop_radius;
    double g;
    double c_gnd, h_clip, c_xy, c_z;
    double dw_c1, dw_c2, dw_c3, dw_max_xy, dw_dz_min;
    double pos_kp[3], pos_ki[3], pos_kd[3], pos_iclamp;
    double att_kp[3], att_ki[3], att_kd[3], att_iclamp;
    double dt_sim, dt_ctrl;
    double sp_rate_pos, sp_rate_yaw;
    int32_t frame;
    int32_t integrator;
    int32_t gnd_heights;
    int32_t controller;
} mdg_constants;

/* Fill *out with the CF2X constants (Table "Drone model parameters", Eq. downwash
 * coefficients, Table "Default PIDControl gains", f_sim = 240 Hz, f_ctrl = 48 Hz) and
 * the project defaults for what the paper does not print: g = 9.81 m/s^2 (MuJoCo's
 * default gravity), c_gnd = 11.36859, c_xy = 9.1785e-7, c_z = 10.311e-7 and
 * h_clip = (r_p/4) sqrt(c_gnd / (T/W - 1)) — the height at which the ground-effect
 * increment at hover thrust equals the spare thrust (T/W - 1) m g, a clip "derived
 * from the propeller radius and the model's maximum thrust" (Section 3.1.3).
 * Host only. Returns MDG_ERR_ARG if out is NULL. */
int mdg_constants_cf2x(mdg_constants* out);
/* CF2P: the CF2X constants with frame = MDG_FRAME_P (Table "Drone model parameters" has
 * one column for both). */
int mdg_constants_cf2p(mdg_constants* out);
/* RACE: the RACE column of Table "Drone model parameters". Not printed for RACE and set
 * here: C_gnd, c_xy, c_z and the downwash coefficients keep their CF2.x values, h_clip
 * follows the CF2X derivation from r_p and T/W, the position gains are kept and the
 * attitude gains are scaled per axis by the inertia ratio J_RACE / J_CF2X. */
int mdg_constants_race(mdg_constants* out);

/* DSLPIDControl (Section 4.2.1: retuned gains, integral clamps halved, setpoint rate
 * limits 2.0 m/s and pi rad/s, feed-forward acceleration) applied to *c in place: the
 * gains are not printed, and are set here by tuning each loop as a second-order system
 * from c's own inertia: position Kp = w^2, Kd = 2 z w, Ki = 0.05 (w = 1.5, 1.5, 2.0 rad/s,
 * z = 0.8, 0.8, 1.0); attitude Kp = J w^2, Kd = 2 z w J, Ki = J (0, 0, 5) (w = 20, 20,
 * 10 rad/s, z = 0.9). pos_iclamp and att_iclamp are halved, controller = MDG_CTRL_DSL.
 * Host only. Returns MDG_ERR_ARG if c is NULL. */
int mdg_controller_dsl(mdg_constants* c);

/* sizeof(mdg_constants), for bindings that mirror the struct. */
int mdg_constants_size(void);

/* HOVER_RPM = sqrt(m g / (4 kf)) and MAX_RPM = sqrt((T/W) m g / (4 kf)) (Section 3.3).
 * Host only; return a negative value for a NULL or non-physical argument. */
double mdg_hover_rpm(const mdg_constants* c);
double mdg_max_rpm(const mdg_constants* c);

/* Create a batch of n_envs environments on the current CUDA device.
 *   drones_per_env  host [n_envs], each in [0, MDG_MAX_ENV_DRONES] (the
 *                   constructor's num_drones per environment, Section 3.4.2)
 *   model_flags     host [n_envs], each a subset of MDG_GND|MDG_DRAG|MDG_DW
 *   c               constants (copied; NULL = mdg_constants_cf2x)
 *   out             receives the handle
 * n_envs = 0 is allowed (every compute call is then a no-op). The handle owns its
 * device tables (CSR offsets, flags, launch tiles, status word); the caller owns
 * every state, action and observation buffer. Errors: MDG_ERR_ARG, MDG_ERR_CUDA. */
int mdg_create(int32_t n_envs, const int32_t* drones_per_env, const uint32_t* model_flags,
               const mdg_constants* c, mdg_handle* out);

/* Release the handle and its device tables (synchronises the device). NULL is allowed. */
int mdg_destroy(mdg_handle h);

/* Number of drones (sum of drones_per_env), or a negative code for a NULL handle. */
int64_t mdg_num_drones(mdg_handle h);

/* Per-environment action types for MDG_ACT_MIXED: host [n_envs], each an action type
 * other than MDG_ACT_MIXED (copied to the device on the default stream, synchronously). */
int mdg_set_action_types(mdg_handle h, const uint8_t* per_env);

/* Attach the DSL controller's setpoints: device float32 [n_drones][4] = (x, y, z, yaw),
 * 16-byte aligned, caller-owned, read and written by every step, rollout, surrogate step
 * and mdg_pid call with the DSL controller (waypoint actions move each drone's setpoint
 * towards its waypoint, rate-limited, and the PID tracks the setpoint). A setpoint whose
 * x is NaN is not set yet and starts at the drone's position and yaw (fill the buffer
 * with NaN to start, or a drone's row to reset it). NULL detaches. Required before any
 * compute call of a handle created with the DSL controller. Errors: MDG_ERR_ARG. */
int mdg_set_setpoints(mdg_handle h, float* setpoints);

/* Attach domain randomization, motor lag, action latency and wind to every step and
 * rollout (all caller-owned device buffers, 16-byte aligned; NULL env_params detaches):
 *   env_params   float32 [n_envs][MDG_DR_PARAMS] (validated here, on a host copy: factors
 *                positive, tau >= 0, delay whole and < hist_depth, known wind bits,
 *                gust probability in [0, 1], durations, altitude positive, noise sigmas
 *                >= 0, sensor delay 0 or 1; change it only by attaching again)
 *   motor        float32 [n_drones][4] rotor speeds, the lag's state (NaN: not set, starts
 *                at the first command)
 *   action_hist  float32 [hist_depth][n_drones][4] actions received (NaN row: empty, filled
 *                with the first action), hist_depth in [1, MDG_MAX_HIST_DEPTH]
 *   wind_state   float32 [n_envs][MDG_WIND_STATE] (start: zeros with the gust phase -1)
 *   seed         of the counter-based wind draws (SplitMix64 over seed, step, environment)
 * Per control step and drone: the action received enters the shift register and the one
 * received `delay` steps ago is applied, through the nominal controller (plane 5 records
 * its RPMs); each motor's command is its RPM times its bias, saturated at MAX_RPM times
 * the factor; the environment's wind (evaluated once per control step) adds its direct
 * force and the quadratic drag on the relative wind at the step's start, held over the
 * substeps; before each substep every rotor speed relaxes towards its command,
 * n <- c + (n - c) exp(-dt_sim/tau); the substeps integrate the randomized model.
 * Observations (the sensor group): with a sensor delay the KIN observation reports the state
 * and RPMs of the step's start; KIN positions, roll/pitch/yaw, velocities and body rates get
 * Gaussian noise of the row's sigmas (counter-based draws keyed by the environment's wind
 * step and the drone); the neighbour observation is neither delayed nor noisy.
 * Euler substeps only (MDG_ERR_UNSUPPORTED with RK4, in mdg_surrogate_step and for
 * observations to host buffers). Errors: MDG_ERR_ARG, MDG_ERR_CUDA (the host copy). */
int mdg_set_randomization(mdg_handle h, const float* env_params, float* motor, float* action_hist,
                          int32_t hist_depth, float* wind_state, uint64_t seed);

/* Episode reset under domain randomization (Section 3.5: the "init" row of Table
 * "Recommended domain-randomization ranges", p0 +-0.2 m, RPY0 +-0.1 rad, v0 +-0.5 m/s, drawn
 * at every reset like the rest of the table, and the "sticky per-episode bias on the
 * observation" of its recommendation (iii), whose size is not printed). For every drone g,
 * from the counter-based generator (SplitMix64 over seed, stream, episode, g, component):
 *   p0   = nominal[g].xyz + init_range[0] (2u - 1) per axis
 *   RPY0 = (0, 0, nominal[g].w) + init_range[1] (2u - 1) per angle, q0 the quaternion of
 *          Rz(yaw) Ry(pitch) Rx(roll)
 *   v0   = init_range[2] (2u - 1) per axis; body rate, PID integrals and last RPMs zero
 * and, when obs_bias is given, obs_bias[g] = 12 Gaussian offsets N(0, bias_sigma[k / 3]^2)
 * for the KIN channels position (k = 0-2), roll/pitch/yaw (3-5), velocity (6-8) and body rate
 * (9-11), which mdg_set_obs_bias makes the observations carry for the episode.
 *   state       device float32 [MDG_STATE_PLANES][n_drones][4], overwritten
 *   nominal     device float32 [n_drones][4] = nominal x, y, z [m] and yaw [rad] (the
 *               constructor's initial_xyzs / initial_rpys, Section 3.4.2)
 *   init_range  host float [3] half-widths (position m, angles rad, velocity m/s), NULL = 0
 *   bias_sigma  host float [4] (position m, angles rad, velocity m/s, body rate rad/s);
 *               required when obs_bias is given
 *   obs_bias    device float32 [n_drones][12] or NULL
 *   seed, episode  the draws' keys: the same pair gives the same episode
 * The randomization's own state (rotor speeds, action history, wind state) and the DSL
 * setpoints are the caller's buffers, reset by the caller (their documented start values).
 * Asynchronous on `stream`. Errors: MDG_ERR_ARG, MDG_ERR_CUDA. */
int mdg_reset(mdg_handle h, float* state, const float* nominal, const float* init_range, const float* bias_sigma,
              float* obs_bias, uint64_t seed, uint64_t episode, void* stream);

/* Attach (or, with NULL, detach) a sticky per-episode observation bias, device float32
 * [n_drones][12] as mdg_reset writes it, 16-byte aligned, caller-owned: every step and
 * rollout under randomization adds it to the KIN observation's position, roll/pitch/yaw,
 * velocity and body rate (on top of the sensor noise, delayed observations included).
 * Requires the randomization to be attached (mdg_set_randomization; attaching it again
 * keeps the bias, detaching it detaches the bias too). Synchronous with the legacy default
 * stream, like mdg_set_randomization. Errors: MDG_ERR_ARG, MDG_ERR_CUDA. */
int mdg_set_obs_bias(mdg_handle h, const float* obs_bias);

/* Threads per block of the step kernels (a multiple of 32 in [32, 1024] and at least
 * the largest environment, rounded up to 32). Environments are packed whole into
 * blocks of at most this many drones. The default (chosen at creation) spreads the
 * blocks evenly over the SMs; mdg_autotune picks by measurement. */
int mdg_set_block_size(mdg_handle h, int32_t threads_per_block);
int32_t mdg_get_block_size(mdg_handle h);

/* One control step (Section 3.4.2: sim_freq/ctrl_freq physics substeps per env.step).
 *   state       device float32 [MDG_STATE_PLANES][n_drones][4], updated in place
 *   action      device float32 [n_drones][4]: RPMs (MDG_ACT_RPM), waypoints
 *               [x, y, z, yaw] (MDG_ACT_PID) or the values of another action type; for
 *               MDG_ACT_MIXED each env reads it according to its type. May be NULL only
 *               when n_drones is 0.
 *   action_type one of the MDG_ACT_* types
 *   n_substeps  >= 1 (5 for 240 Hz physics at 48 Hz control)
 * The action is turned into four RPMs once (PID, VEL, ATTITUDE: Section 4.2.1, updating
 * the integrals in planes 3-4), held for n_substeps substeps of dt_sim, and recorded in
 * plane 5. Within a substep every drone of an environment sees the positions of the
 * others at the start of that substep. A non-finite result sets MDG_STATUS_NONFINITE.
 * Errors: MDG_ERR_ARG (bad pointer/alignment/type/count, MIXED without types),
 * MDG_ERR_CUDA (launch failure). */
int mdg_step(mdg_handle h, float* state, const float* action, int32_t action_type, int32_t n_substeps,
             void* stream);

/* mdg_step followed, in the same kernel, by the observations of the new state
 * (the outputs of mdg_obs). kin and nbr_idx are required; nbr_rel may be NULL. */
int mdg_step_obs(mdg_handle h, float* state, const float* action, int32_t action_type, int32_t n_substeps,
                 float* kin, int32_t* nbr_idx, float* nbr_rel, void* stream);

/* mdg_step_obs with the actions read from, and the observations written to, page-locked
 * host memory that the device can address (cudaHostAlloc, or cudaHostRegister with
 * cudaHostRegisterMapped): the step kernel itself loads the actions and stores the
 * observations across the host link, so the transfers overlap its arithmetic and no
 * separate copies are issued. The state stays in device memory. This is the call for a
 * host-side consumer of every step (a learner, a logger); the paper's environment returns
 * observations to the host after every step in the same way (Section 3.4.2).
 *   state                  as for mdg_step (device memory)
 *   action_host            page-locked float32 [n_drones][4], 16-byte aligned
 *   kin_host, nbr_idx_host, nbr_rel_host (may be NULL)   page-locked, layouts of mdg_obs
 * The outputs are complete once `stream` has passed the step (synchronise on it or on an
 * event recorded after the call before reading them).
 * Errors: MDG_ERR_ARG when a buffer is not mapped page-locked host memory or as
 * mdg_step_obs; MDG_ERR_CUDA. */
int mdg_step_obs_host(mdg_handle h, float* state, const float* action_host, int32_t action_type, int32_t n_substeps,
                      float* kin_host, int32_t* nbr_idx_host, float* nbr_rel_host, void* stream);

/* The PID controller alone (PIDControl.computeControl, Section 4.2.1): for every
 * drone, from its state and waypoint [x, y, z, yaw], the four RPMs, the position
 * error and the yaw error; the integrals in state planes 3-4 are updated in place.
 *   state      device float32 [MDG_STATE_PLANES][n_drones][4] (planes 3-4 written)
 *   waypoints  device float32 [n_drones][4]
 *   rpm_out    device float32 [n_drones][4]
 *   pos_err    device float32 [n_drones][3] or NULL
 *   yaw_err    device float32 [n_drones] or NULL */
int mdg_pid(mdg_handle h, float* state, const float* waypoints, float* rpm_out, float* pos_err, float* yaw_err,
            void* stream);

/* mdg_pid with a feed-forward acceleration (DSLPIDControl's target_acc, added to the
 * position loop's output before the thrust direction is formed; any controller):
 *   target_acc device float32 [n_drones][4] = (a_x, a_y, a_z, unused) [m/s^2], or NULL
 *              (zero). The step functions' waypoint actions carry no feed-forward. */
int mdg_pid_ff(mdg_handle h, float* state, const float* waypoints, const float* target_acc, float* rpm_out,
               float* pos_err, float* yaw_err, void* stream);

/* Camera frames (Section 3.4.4, the RGB observation: (48, 64, 4) uint8 from each drone's
 * onboard camera, 60 degree field of view, at [0.02, 0, 0] in the body frame), ray cast from
 * primitive shapes since no renderer or meshes are used. Readings: pinhole camera along body
 * +x (image right = body -y, up = body +z), 60 degrees the vertical field of view, pixels
 * through their cell centres, row 0 on top; the environment's other drones as oblate
 * ellipsoids in their body frames with semi-axes (L + r_p, L + r_p, 0.3 (L + r_p)); the
 * ground z = 0 as a 0.5 m checkerboard (greys 0.55 / 0.35) seen from above; the camera's
 * own drone not drawn; Lambert shading ambient 0.35 + diffuse 0.65 max(0, n . l), l along
 * (0.3, 0.2, 1); drone k coloured by an 8-entry palette (k mod 8); sky (0.55, 0.70, 0.90);
 * channels round(255 c), alpha 255. Outputs (each may be NULL; device, 4-byte aligned):
 *   rgba   uint8 [n_drones][MDG_CAM_H][MDG_CAM_W][4]
 *   depth  float32 [n_drones][MDG_CAM_H][MDG_CAM_W]: distance along the optical axis to the
 *          nearest surface beyond 1e-4 m, +inf where only sky is seen
 *   seg    int32 [n_drones][MDG_CAM_H][MDG_CAM_W]: -1 sky, 0 ground, 1 + global drone index
 * Errors: MDG_ERR_ARG, MDG_ERR_CUDA. */
#define MDG_CAM_H 48
#define MDG_CAM_W 64
int mdg_render(mdg_handle h, const float* state, uint8_t* rgba, float* depth, int32_t* seg, void* stream);

/* Observations of the current state (Section 3.4.4 KIN, and the neighbourhood
 * adjacency of the abstract):
 *   kin      device float32 [n_drones][20]: p, q, roll/pitch/yaw (ZYX), v, w, a_prev
 *   nbr_idx  device int32 [n_drones][4]: global indices of the 4 nearest other drones
 *            of the same environment (Euclidean distance, ties to the lower index),
 *            -1 where the environment has fewer than 5 drones; a drone whose squared
 *            distance is not finite (a NaN or infinite position) is not listed
 *   nbr_rel  device float32 [n_drones][24] or NULL: per neighbour [p_i - p_j, v_i - v_j],
 *            zeros for padded slots */
int mdg_obs(mdg_handle h, const float* state, float* kin, int32_t* nbr_idx, float* nbr_rel, void* stream);

/* Observation modes of mdg_rollout. */
#define MDG_OBS_NONE 0       /* no observations */
#define MDG_OBS_LAST 1       /* observations of the state after the last step ([n] outputs) */
#define MDG_OBS_EVERY_STEP 2 /* observations after every step ([K][n] outputs) */

/* K control steps in one launch (uneven batches in one persistent launch). Persistent
 * thread blocks take work items — whole environments, for uneven batches grouped after
 * sorting the environments by (size, physics subset) so that a warp's environments share
 * both — from an atomic counter, longest items first, and advance each item through all
 * K steps with the drones' state in registers: the state is read and written once per
 * rollout. Every step is exactly mdg_step's (Section 3.4.2 per step), so K calls of
 * mdg_step_obs give the same result.
 *   state            as for mdg_step (updated in place)
 *   actions          device float32 [K][n_drones][4] when action_per_step != 0, else one
 *                    [n_drones][4] used for every step (e.g. fixed PID waypoints)
 *   action_type, n_substeps   as for mdg_step
 *   K                number of control steps (0: no-op)
 *   obs_mode         MDG_OBS_NONE / MDG_OBS_LAST / MDG_OBS_EVERY_STEP; kin, nbr_idx and
 *                    nbr_rel (may be NULL) are laid out as for mdg_obs, with a leading
 *                    [K] dimension for MDG_OBS_EVERY_STEP
 * The handle owns the work counter, so rollouts of one handle must not overlap on the GPU.
 * Errors: as mdg_step. */
int mdg_rollout(mdg_handle h, float* state, const float* actions, int32_t action_per_step, int32_t action_type,
                int32_t n_substeps, int32_t K, int32_t obs_mode, float* kin, int32_t* nbr_idx, float* nbr_rel,
                void* stream);

/* A CUDA graph of one mdg_rollout with fixed arguments (the work-counter reset and the
 * persistent launch), for replaying a K-step rollout with one host call. The buffers are
 * bound at creation; the graph is tied to the handle's device and to its current block
 * size (create it after mdg_autotune / mdg_set_block_size). Launch it on any stream. */
typedef struct mdg_graph_s* mdg_graph;
int mdg_rollout_graph_create(mdg_handle h, float* state, const float* actions, int32_t action_per_step,
                             int32_t action_type, int32_t n_substeps, int32_t K, int32_t obs_mode, float* kin,
                             int32_t* nbr_idx, float* nbr_rel, mdg_graph* out);
int mdg_graph_launch(mdg_graph g, void* stream);
int mdg_graph_destroy(mdg_graph g);

/* Work distribution of the persistent rollout kernel (mdg_rollout and its graphs):
 *   mode         MDG_SCHED_DYNAMIC (default): the blocks take the work items, longest first,
 *                from an atomic counter, so each launch may hand them out in another order;
 *                MDG_SCHED_STATIC: a fixed schedule built on the host, longest processing time
 *                first (items by decreasing estimated chain, each to the block with the least
 *                estimated work), the same every launch
 *   item_drones  uneven batches: at most this many drones per work item (environments are
 *                packed whole; one larger than this is an item of its own); 0 = the block size.
 *                Smaller items give the schedule finer pieces to balance.
 * Host only; takes effect at the next rollout (graphs capture the tables of their creation).
 * Errors: MDG_ERR_ARG. */
#define MDG_SCHED_DYNAMIC 0
#define MDG_SCHED_STATIC 1
int mdg_set_rollout_schedule(mdg_handle h, int32_t mode, int32_t item_drones);
int mdg_get_rollout_schedule(mdg_handle h, int32_t* mode, int32_t* item_drones);

/* Autotuner: times the step kernels (K = 0: mdg_step_obs; K > 0: a K-step mdg_rollout
 * with observations after the last step) on the caller's state and actions for every
 * block size 32, 64, 128, ..., 1024 that holds the largest environment and, for rollouts,
 * both schedules of mdg_set_rollout_schedule and (uneven batches) the item caps of the whole
 * block, half and a quarter of it (at least the largest environment and 32 drones): 5 timed
 * launches after 2 warm-ups each, the state restored before every launch. Keeps the fastest
 * combination (mdg_set_block_size, mdg_set_rollout_schedule) and restores the state.
 * Allocates temporary scratch; synchronises `stream`. Writes the chosen block size and its
 * mean time in ms (either pointer may be NULL; mdg_get_rollout_schedule reads the rest). */
int mdg_autotune(mdg_handle h, float* state, const float* actions, int32_t action_per_step, int32_t action_type,
                 int32_t n_substeps, int32_t K, void* stream, int32_t* best_block, float* best_ms);

/* Read and clear the status word: synchronises `stream`, writes the MDG_STATUS_* bits
 * raised since the last call to *bits and the smallest offending drone index (or -1)
 * to *first_drone (either may be NULL). Returns MDG_ERR_NONFINITE if the non-finite
 * bit was set, else MDG_OK (or MDG_ERR_CUDA). */
int mdg_status(mdg_handle h, void* stream, uint32_t* bits, int64_t* first_drone);

/* Wait on the host for `stream` to finish its work, for at most timeout_ms milliseconds
 * (polling, so the calling thread never blocks inside the driver). Returns MDG_OK when the
 * stream is idle, MDG_ERR_TIMEOUT when the limit ran out first (the work keeps running; the
 * caller decides whether to wait again, report a stuck worker or tear down), MDG_ERR_CUDA
 * when the stream reports an error, MDG_ERR_ARG for a negative limit. The paper's
 * environments step synchronously (Section 3.4.2); this is the bounded form of that wait
 * for a host loop that must notice a stuck device. */
int mdg_sync(void* stream, int32_t timeout_ms);

/* One control step that allocates no device memory: mdg_step_obs (or mdg_step when
 * kin is NULL) for a batch described on the host, with no handle. The paper has no
 * counterpart; this entry point exists for callers that cannot call cudaMalloc, for
 * example a process whose device memory is owned by another allocator (a training
 * framework's caching allocator that has reserved the free memory) or a control loop
 * that must not allocate after it starts. mdg_create allocates the batch tables and the
 * status word, so such callers cannot hold a handle.
 *
 * Instead of allocating, the call keeps the batch tables (CSR offsets, physics flags,
 * action types, launch tiles) and the status word in one file-scope static device array
 * of MDG_NOALLOC_SCRATCH_BYTES (about 353 KiB), which every GPU that loads the library
 * holds until the process exits. It supports at most MDG_NOALLOC_MAX_ENVS environments
 * and rejects larger batches with MDG_ERR_ARG. The caller passes every input and output:
 *   c               constants (NULL = mdg_constants_cf2x)
 *   n_envs, drones_per_env, model_flags   host arrays, as for mdg_create
 *   action_types    host [n_envs] RPM/PID per environment when action_type is
 *                   MDG_ACT_MIXED, else ignored (may be NULL)
 *   state, action, action_type, n_substeps, kin, nbr_idx, nbr_rel   as for mdg_step_obs
 *                   (kin = NULL: no observations, nbr_idx and nbr_rel are ignored)
 *   status_out      device uint32 [2] or NULL: receives this call's status bits and the
 *                   smallest non-finite drone index (0xffffffff if none), as mdg_status
 *                   reports them; not written when the batch has no drones
 * Each call uploads the tables and a cleared status word into the array with
 * cudaMemcpyAsync on `stream` from a static host staging buffer, then launches the step
 * kernel there. It calls no cudaMalloc, cudaFree or other allocating routine.
 * Every call looks up the array's device address with the device current. The first call
 * on a device also loads the library's device code there (lazy module loading, the CUDA
 * default), which reserves the array and the code in that device's memory: make it before
 * another allocator takes the device's free memory (it fails with MDG_ERR_CUDA and a
 * message naming this cause otherwise). All calls share the array and it keeps the last
 * call's contents, so calls that overlap on the GPU (on different streams or from
 * different host threads) race; serialise them. A call made while `stream` is being
 * captured into a CUDA graph returns MDG_ERR_UNSUPPORTED: the tables come from a host
 * staging buffer that the next call overwrites, so a replay would read another batch's
 * tables. Errors: MDG_ERR_ARG (as mdg_create / mdg_step_obs, or too many environments),
 * MDG_ERR_UNSUPPORTED (DSL controller, stream capture), MDG_ERR_CUDA. */
#define MDG_NOALLOC_MAX_ENVS 16384
#define MDG_NOALLOC_SCRATCH_BYTES 360960
int mdg_step_obs_noalloc(const mdg_constants* c, int32_t n_envs, const int32_t* drones_per_env,
                         const uint32_t* model_flags, const uint8_t* action_types, float* state, const float* action,
                         int32_t action_type, int32_t n_substeps, float* kin, int32_t* nbr_idx, float* nbr_rel,
                         uint32_t* status_out, void* stream);

/* ---- learned surrogate (not in the paper) ----
 * A multilayer perceptron stands in for the substep loop of one control step: from a
 * drone's 13-d state (p, q, v, w), its four RPMs and its 4 nearest neighbours' relative
 * positions and velocities (41 inputs) it predicts the 13-d state change over the control
 * step. 41 -> 256 -> 256 -> 256 -> 13, SiLU hidden activations, bfloat16 weights and
 * activations with FP32 accumulation on the tensor cores, trained with Adam on MSE of
 * standardised targets. Stored padded: 64 inputs, 32 outputs (zeros beyond 41 / 13).
 * Flat FP32 parameter layout (MDG_MLP_PARAMS floats): W1 [256][64], b1 [256],
 * W2 [256][256], b2, W3 [256][256], b3, W4 [32][256], b4 [32]. */
#define MDG_MLP_IN 41
#define MDG_MLP_IN_PAD 64
#define MDG_MLP_HIDDEN 256
#define MDG_MLP_OUT 13
#define MDG_MLP_OUT_PAD 32
#define MDG_MLP_PARAMS 156448

typedef struct mdg_mlp_s* mdg_mlp;

/* Create a surrogate on the current device with scratch for batches of up to max_batch
 * rows (a positive multiple of 128). init: host FP32 [MDG_MLP_PARAMS] or NULL (zeros). */
int mdg_mlp_create(int32_t max_batch, const float* init, mdg_mlp* out);
int mdg_mlp_destroy(mdg_mlp m);
/* Copy the FP32 master parameters (or the last computed gradients) to/from the host
 * (flat layout above; synchronous). */
int mdg_mlp_get_params(mdg_mlp m, float* host_out);
int mdg_mlp_set_params(mdg_mlp m, const float* host_in);
int mdg_mlp_get_grads(mdg_mlp m, float* host_out);
/* Input standardisation (41 means and standard deviations), output de-standardisation
 * (13), and the out-of-distribution box of the raw inputs (41 lower and upper bounds);
 * host arrays, copied. */
int mdg_mlp_set_normalization(mdg_mlp m, const float* in_mean, const float* in_std, const float* out_mean,
                              const float* out_std, const float* in_lo, const float* in_hi);
/* x = bf16((raw - mean) / std), raw device [rows][41] FP32, x device [rows][64] bf16 (uint16). */
int mdg_mlp_standardize(mdg_mlp m, const float* raw, uint16_t* x, int64_t rows, void* stream);
/* Forward pass: x device [B][64] bf16, y device [B][32] FP32 (standardised outputs);
 * B a multiple of 128, at most max_batch. On MDG_MLP_PATH_TCGEN05_PAIRS x is read by TMA
 * (a tensor map over [B][64]) and must be 16-byte aligned (else MDG_ERR_CUDA). */
int mdg_mlp_forward(mdg_mlp m, const uint16_t* x, float* y, int32_t B, void* stream);
/* Gradient of the MSE between the forward output and the standardised targets
 * t device [B][32] (columns 13..31 ignored) into the surrogate's gradient buffer;
 * loss_out: device float or NULL (receives the loss). */
int mdg_mlp_grad(mdg_mlp m, const uint16_t* x, const float* t, int32_t B, float* loss_out, void* stream);
/* One Adam step (b1 0.9, b2 0.999, eps 1e-8) with the gradient of the last mdg_mlp_grad. */
int mdg_mlp_adam(mdg_mlp m, float lr, void* stream);

/* Inference path of mdg_mlp_forward and mdg_surrogate_step: MDG_MLP_PATH_TCGEN05_PAIRS
 * (default), MDG_MLP_PATH_TCGEN05 (one fused kernel on tcgen05.mma with the accumulator in
 * tensor memory and the activations in shared memory, one 128-row tile in flight per block)
 * or MDG_MLP_PATH_MMA_SYNC (one mma.sync GEMM per layer, the training kernels). Training has
 * its own setting, mdg_mlp_set_train_path. */
#define MDG_MLP_PATH_MMA_SYNC 0
#define MDG_MLP_PATH_TCGEN05 1
/* MDG_MLP_PATH_TCGEN05_PAIRS: the fused tcgen05 kernel with two 128-row tiles in flight per
 * block (each layer's accumulator is moved to registers before its SiLU, so one tile needs one
 * 256-column accumulator and the tensor cores run one tile while the epilogue works on the
 * other; the second tile of a pair reuses two of the first tile's four weight chunks per
 * hidden layer and sums its K chunks in another order, so its outputs agree with the
 * single-tile kernel to FP32 summation order, the first tile's bit for bit). Inference only;
 * training uses mdg_mlp_set_train_path. */
#define MDG_MLP_PATH_TCGEN05_PAIRS 2
int mdg_mlp_set_path(mdg_mlp m, int32_t path);
/* Training path of mdg_mlp_grad: MDG_MLP_PATH_TCGEN05 (default: every GEMM of the forward and
 * backward pass on tcgen05.mma with the accumulator in tensor memory, both operands K-major in
 * shared memory; the epilogues write the pre-activations, the SiLU activations and the
 * hidden gradients together with their transposes, which are the K-major operands of the
 * weight gradients dW = dZ^T X; those are split over the batch and added up with atomics) or
 * MDG_MLP_PATH_MMA_SYNC (the mma.sync GEMMs). Errors: MDG_ERR_ARG. */
int mdg_mlp_set_train_path(mdg_mlp m, int32_t path);
/* Bounds of the tcgen05 kernel's waits on its own mbarriers (its MMAs, bulk copies and
 * epilogue hand-offs): try_waits mbarrier.try_wait calls (each suspends at most ~1 us) for
 * the producer and MMA waits, polls test_wait polls for the MMA/epilogue hand-offs; a wait
 * that runs out sets MDG_STATUS_TIMEOUT, and the kernel then abandons its tiles: every role
 * leaves its loop, the copies and MMAs already issued are waited for with the default bound,
 * the tensor memory is freed and the launch returns (outputs of abandoned tiles are not
 * written). For exercising that exit without a stuck device: 0 gives up at the first wait
 * that is not already complete. A negative value restores the default (the constants below,
 * a few tenths of a second each). Host only; affects later launches of this surrogate. */
#define MDG_MLP_DEFAULT_TRY_WAITS 262144
#define MDG_MLP_DEFAULT_POLLS 4194304
int mdg_mlp_set_wait_limits(mdg_mlp m, int32_t try_waits, int32_t polls);
/* Read and clear the surrogate's status word (synchronises `stream`): MDG_STATUS_TIMEOUT
 * if a tensor-core kernel abandoned its work. */
int mdg_mlp_status(mdg_mlp m, void* stream, uint32_t* bits);

/* One transition of the plain integrator, the surrogate's training data: the RPMs applied
 * (applied = rpm times rpm_scale elementwise, or rpm when rpm_scale is NULL; device
 * [n_drones][4], written), the raw inputs of the current state with them (as mdg_features),
 * one control step of n_substeps with them as RPM actions (the state advances in place), and
 * the 13-d state change delta = [p, q, v, w] after minus before (device [n_drones][13]).
 * rpm, rpm_scale, applied and state 16-byte aligned. Errors: as mdg_step, mdg_features. */
int mdg_transition(mdg_handle h, float* state, const float* rpm, const float* rpm_scale, float* applied, float* raw,
                   float* delta, int32_t n_substeps, void* stream);

/* Standardisation of a set of N transitions (raw device [N][41], delta device [N][13]) for
 * training, and the surrogate's normalisation from it (as mdg_mlp_set_normalization):
 *  1. rows with a non-finite value are dropped;
 *  2. trim box: per column the quantiles trim_frac and 1 - trim_frac (linear interpolation
 *     between order statistics) over an evenly strided sample of at most 262144 finite rows,
 *     widened on each side by margin times their distance; rows outside the box in any column
 *     are dropped (the chaotic tail of near-coincident downwash heights lives there);
 *  3. mean and standard deviation (FP64, unbiased) of every column over the kept rows; a
 *     column whose deviation is below 1e-6 max(|mean|, 1) is scaled by 1;
 *  4. rows with a standardised input beyond +-ood_z or a standardised target beyond
 *     +-target_clip are dropped;
 *  5. out-of-distribution box: the kept inputs' range, widened by 10% of it plus 1e-6;
 *  6. the kept rows, in their order, truncated to a multiple of 128: x_out device [N][64]
 *     bf16 (uint16) standardised inputs (zero padded), t_out device [N][32] standardised
 *     targets (zero padded); *n_kept receives their number, *n_finite the rows of step 1.
 * Allocates temporary device scratch and synchronises `stream`.
 * Errors: MDG_ERR_ARG (bad arguments, too few usable rows), MDG_ERR_CUDA. */
int mdg_mlp_fit_normalization(mdg_mlp m, const float* raw, const float* delta, int64_t N, float trim_frac, float margin,
                              float ood_z, float target_clip, uint16_t* x_out, float* t_out, int64_t* n_finite,
                              int64_t* n_kept, void* stream);
/* The normalisation in use (host arrays: 41 input means, standard deviations, box lower and
 * upper bounds; 13 output means and standard deviations; any pointer may be NULL). */
int mdg_mlp_get_normalization(mdg_mlp m, float* in_mean, float* in_std, float* out_mean, float* out_std, float* in_lo,
                              float* in_hi);

/* Raw surrogate inputs of the current state: raw device [n_drones][41] =
 * [p, q, v, w, rpm (4), 4 nearest neighbours' (p_i - p_j, v_i - v_j)]; rpm device
 * [n_drones][4] are the RPMs to be applied. */
int mdg_features(mdg_handle h, const float* state, const float* rpm, float* raw, void* stream);

/* One control step with the surrogate in place of the substep loop (uniform batches: every
 * environment of one size; n_drones <= the surrogate's max_batch): the action
 * becomes RPMs as in mdg_step (PID integrals and plane 5 updated), the inputs are
 * standardised, the network predicts the state change, q is renormalised. An environment
 * any of whose drones has a standardised input beyond +-ood_z or a raw input outside the
 * normalisation box takes the plain integrator instead (n_substeps substeps of the handle's
 * integrator, Euler or RK4, with the handle's physics). On MDG_MLP_PATH_TCGEN05_PAIRS (the
 * default) the network kernel adds the de-standardised change to the state itself; the other
 * paths write the network's outputs and a separate kernel adds them (same arithmetic).
 * n_fallback: device int32 or NULL, receives the number of such environments. */
int mdg_surrogate_step(mdg_handle h, mdg_mlp m, float* state, const float* action, int32_t action_type,
                       int32_t n_substeps, float ood_z, int32_t* n_fallback, void* stream);

/* Message of the last error on this host thread ("" if none). */
const char* mdg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MDG_H */
