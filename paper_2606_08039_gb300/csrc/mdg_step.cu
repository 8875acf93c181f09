// Step, PID and observation kernels of the batched Crazyflie dynamics (sm_103a).
//
// One thread owns one drone for a whole control step: its 13-float state, its PID
// integrals and its four RPMs stay in registers across the substeps. A thread block
// holds whole environments (a "tile" built on the host), so the inter-drone downwash
// of Eq. downwash only needs the block's shared memory: every substep each thread
// publishes its position into a double-buffered shared array, one barrier makes the
// start-of-substep snapshot visible, and each drone sums the wake of the drones of its
// own environment from shared memory. State moves between HBM and registers once per
// control step, as coalesced float4 planes.
#include <cuda_bf16.h>
#include <math.h>

#include "mdg.h"
#include "mdg_internal.cuh"

namespace mdg {
namespace {

constexpr float kPi = 3.14159265358979323846f;

// Approximate reciprocal and base-2 exponential of the special function unit
// (rcp.approx.ftz.f32: relative error within 2^-23; ex2.approx.ftz.f32: within 2^-22).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Square root of the special function unit (sqrt.approx.ftz.f32, relative error near
// 2^-23): the RPMs and the collective thrust of the controllers, outputs that no later
// rounding depends on.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// atan2 by reduction to a = min(|x|, |y|) / max(|x|, |y|) in [0, 1], then the octant:
// atan(a) is the odd polynomial a P(a^2), P of degree 7, a near-minimax fit of the absolute
// error on [0, 1] (Lawson's iteratively reweighted least squares; fit_atan.py beside this
// file prints the coefficients and checks them): |error| below 1.4e-7 rad in float32, plus
// the reciprocal's 2^-23. Signs of zeros as in C (the sign bit of x picks the half plane).
// NaN in, NaN out; both |x| and |y| below 2^-126 give an angle of the right quadrant only.
__device__ __forceinline__ float atan2_fast(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float a = mn * rcp_approx(fmaxf(mx, 1.17549435e-38f));
    const float s = a * a;
    float p = fmaf(s, -0.00405449513f, 0.0218627099f);
    p = fmaf(p, s, -0.0559119843f);
    p = fmaf(p, s, 0.0964217335f);
    p = fmaf(p, s, -0.139086202f);
    p = fmaf(p, s, 0.199465647f);
    p = fmaf(p, s, -0.333298594f);
    p = fmaf(p, s, 0.999999344f);
    float r = a * p;
    r = ay > ax ? 1.57079637f - r : r;
    r = __float_as_int(x) < 0 ? 3.14159274f - r : r;
    r = copysignf(r, y);
    const float t = ax + ay;
    return t != t ? t : r;
}

// asin(s) for s in [-1, 1] as atan2(s, sqrt((1 - s)(1 + s))).
__device__ __forceinline__ float asin_fast(float s)
{
    return atan2_fast(s, sqrt_approx((1.f - s) * (1.f + s)));
}

// An angle reduced by a multiple of 2 pi to about [-pi, pi]: Cody and Waite's reduction
// (2 pi = c_hi + c_lo, c_hi the float nearest 2 pi, c_lo the float nearest the remainder),
// within a few 1e-7 rad of the exact remainder for |x| up to ~1e5 rad, where a float32
// difference x - y would already have lost the ulp of x.
__device__ __forceinline__ float reduce_angle(float x)
{
    const float k = rintf(x * 0.159154943f);
    return fmaf(-k, -1.74845553e-7f, fmaf(-k, 6.28318548f, x));
}

// sin and cos of an angle reduced to [-pi, pi], where the special function unit's sine and
// cosine are within 2^-21.4 absolute.
__device__ __forceinline__ void sincos_reduced(float x, float* s, float* c)
{
    __sincosf(reduce_angle(x), s, c);
}

struct Drone {
    float p[3], q[4], v[3], w[3];
    float ip[3], ia[3];  // PID position / attitude error integrals
};

struct Motor {
    float T, tau[3], wsum;  // collective thrust, body torques, 2 pi/60 * sum of RPMs
};

__device__ __forceinline__ void load_state(const float4* __restrict__ S, long long n, long long g, Drone& d,
                                           bool att_int)
{
    const float4 a = S[g], b = S[n + g], c = S[2 * n + g], e = S[3 * n + g];
    d.p[0] = a.x; d.p[1] = a.y; d.p[2] = a.z;
    d.q[0] = a.w; d.q[1] = b.x; d.q[2] = b.y; d.q[3] = b.z;
    d.v[0] = b.w; d.v[1] = c.x; d.v[2] = c.y;
    d.w[0] = c.z; d.w[1] = c.w; d.w[2] = e.x;
    d.ip[0] = e.y; d.ip[1] = e.z; d.ip[2] = e.w;
    if (att_int) {
        const float4 f = S[4 * n + g];
        d.ia[0] = f.x; d.ia[1] = f.y; d.ia[2] = f.z;
    } else {
        d.ia[0] = d.ia[1] = d.ia[2] = 0.f;
    }
}

__device__ __forceinline__ void unpack_state(const float4& a, const float4& b, const float4& c, const float4& e,
                                             const float4& f, Drone& d)
{
    d.p[0] = a.x; d.p[1] = a.y; d.p[2] = a.z;
    d.q[0] = a.w; d.q[1] = b.x; d.q[2] = b.y; d.q[3] = b.z;
    d.v[0] = b.w; d.v[1] = c.x; d.v[2] = c.y;
    d.w[0] = c.z; d.w[1] = c.w; d.w[2] = e.x;
    d.ip[0] = e.y; d.ip[1] = e.z; d.ip[2] = e.w;
    d.ia[0] = f.x; d.ia[1] = f.y; d.ia[2] = f.z;
}

__device__ __forceinline__ void store_state(float4* __restrict__ S, long long n, long long g, const Drone& d,
                                            bool att_int)
{
    S[g] = make_float4(d.p[0], d.p[1], d.p[2], d.q[0]);
    S[n + g] = make_float4(d.q[1], d.q[2], d.q[3], d.v[0]);
    S[2 * n + g] = make_float4(d.v[1], d.v[2], d.w[0], d.w[1]);
    S[3 * n + g] = make_float4(d.w[2], d.ip[0], d.ip[1], d.ip[2]);
    if (att_int) S[4 * n + g] = make_float4(d.ia[0], d.ia[1], d.ia[2], 0.f);
}

// Roll, pitch, yaw in the ZYX convention.
__device__ __forceinline__ void rpy_of(const float q[4], float& roll, float& pitch, float& yaw)
{
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    roll = atan2_fast(2.f * (w * x + y * z), 1.f - 2.f * (x * x + y * y));
    pitch = asin_fast(fminf(1.f, fmaxf(-1.f, 2.f * (w * y - z * x))));
    yaw = atan2_fast(2.f * (w * z + x * y), 1.f - 2.f * (y * y + z * z));
}

// Eq. motor, X configuration: F_i = k_f n_i^2, T = sum F_i,
// tau_x = L/sqrt2 (F0 + F1 - F2 - F3), tau_y = L/sqrt2 (-F0 + F1 + F2 - F3),
// tau_z = k_m (-n0^2 + n1^2 - n2^2 + n3^2). The RPMs are fixed over the control step,
// so this runs once per control step.
__device__ __forceinline__ Motor motor(const float n[4], const DevConsts& c)
{
    const float n0 = n[0] * n[0], n1 = n[1] * n[1], n2 = n[2] * n[2], n3 = n[3] * n[3];
    const float f0 = c.kf * n0, f1 = c.kf * n1, f2 = c.kf * n2, f3 = c.kf * n3;
    Motor m;
    m.T = (f0 + f1) + (f2 + f3);
    if (c.frame_p) {  // + layout: rotors at L (+x, +y, -x, -y)
        m.tau[0] = c.l_sqrt2 * (f1 - f3);
        m.tau[1] = c.l_sqrt2 * (f2 - f0);
    } else {
        m.tau[0] = c.l_sqrt2 * ((f0 + f1) - (f2 + f3));
        m.tau[1] = c.l_sqrt2 * ((f1 + f2) - (f0 + f3));
    }
    m.tau[2] = c.km * ((n1 + n3) - (n0 + n2));
    m.wsum = c.drag_k * ((n[0] + n[1]) + (n[2] + n[3]));
    return m;
}

// Cascaded PID of Section 4.2.1 (position PID -> T = m |a*| and small-angle attitude
// target -> attitude PID -> inverse mixing). The X mixing rows [1,1,1,1], [1,1,-1,-1],
// [-1,1,1,-1], [-1,1,-1,1] are mutually orthogonal with squared norm 4, so the solve of
// M f = [T, tau] is f = 1/4 (T + sqrt2/L tau_x r1 + sqrt2/L tau_y r2 + k_f/k_m tau_z r3);
// for the + layout the rows [0,1,0,-1] and [-1,0,1,0] (norm^2 2, times L^2) give
// f = 1/4 (T + 2/L tau_x r1 + 2/L tau_y r2 + k_f/k_m tau_z r3). r1, r2 are mix_x, mix_y.
template <bool kRate>
__device__ __forceinline__ void attitude_and_mix(Drone& d, float T, float phi_t, float theta_t, float psi_t, float wz_t,
                                                 float roll, float pitch, float yaw, const DevConsts& c, float rpm[4],
                                                 float& yaw_err)
{
    float e[3] = {phi_t - roll, theta_t - pitch, psi_t - yaw};
    e[2] -= 2.f * kPi * floorf((e[2] + kPi) * (0.5f / kPi));  // wrap to [-pi, pi)
    float tau[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        d.ia[r] = fminf(c.att_iclamp, fmaxf(-c.att_iclamp, d.ia[r] + e[r] * c.dt_ctrl));
        tau[r] = c.att_kp[r] * e[r] + c.att_ki[r] * d.ia[r] - c.att_kd[r] * d.w[r];
    }
    if (kRate)  // target body rate [0, 0, wz_t]
        tau[2] = c.att_kp[2] * e[2] + c.att_ki[2] * d.ia[2] + c.att_kd[2] * (wz_t - d.w[2]);
    const float tx = tau[0] * c.alloc_xy, ty = tau[1] * c.alloc_xy, tz = tau[2] * c.alloc_z;
    // multiplying by the signs +-1, 0 is exact, so the X layout rounds as T + tx - ty - tz
    const float f[4] = {0.25f * (((T + c.mix_x[0] * tx) + c.mix_y[0] * ty) - tz),
                        0.25f * (((T + c.mix_x[1] * tx) + c.mix_y[1] * ty) + tz),
                        0.25f * (((T + c.mix_x[2] * tx) + c.mix_y[2] * ty) - tz),
                        0.25f * (((T + c.mix_x[3] * tx) + c.mix_y[3] * ty) + tz)};
#pragma unroll
    for (int i = 0; i < 4; ++i) rpm[i] = sqrt_approx(fminf(c.f_max, fmaxf(0.f, f[i])) * c.inv_kf);
    yaw_err = e[2];
}

// kFF: add the feed-forward acceleration ff (DSLPIDControl's target_acc) to the position
// loop's output (the standalone controller only; waypoint actions carry none). rpy_known:
// the drone's roll, pitch and yaw when the caller already has them for this state.
template <bool kFF = false>
__device__ __forceinline__ void pid(Drone& d, const float4 wp, const DevConsts& c, float rpm[4], float ep[3],
                                    float& yaw_err, float4 ff = float4{}, const float* rpy_known = nullptr)
{
    const float tgt[3] = {wp.x, wp.y, wp.z};
    const float aff[3] = {ff.x, ff.y, ff.z};
    float acc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        ep[r] = tgt[r] - d.p[r];
        d.ip[r] = fminf(c.pos_iclamp, fmaxf(-c.pos_iclamp, d.ip[r] + ep[r] * c.dt_ctrl));
        acc[r] = c.pos_kp[r] * ep[r] + c.pos_ki[r] * d.ip[r] - c.pos_kd[r] * d.v[r];
        if (kFF) acc[r] += aff[r];
    }
    acc[2] += c.g;
    const float T = c.mass * sqrt_approx(acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2]);
    // the target yaw reduced once: its sine and cosine and the yaw error (wrapped again in
    // attitude_and_mix) both take the reduced angle
    const float psi_t = reduce_angle(wp.w);
    float sps, cps;
    __sincosf(psi_t, &sps, &cps);
    const float phi_t = (acc[0] * sps - acc[1] * cps) * c.inv_g;
    const float theta_t = (acc[0] * cps + acc[1] * sps) * c.inv_g;
    float roll, pitch, yaw;
    if (rpy_known) {
        roll = rpy_known[0], pitch = rpy_known[1], yaw = rpy_known[2];
    } else {
        rpy_of(d.q, roll, pitch, yaw);
    }
    attitude_and_mix<false>(d, T, phi_t, theta_t, psi_t, 0.f, roll, pitch, yaw, c, rpm, yaw_err);
}

// DSLPIDControl's setpoint limiter (Section 4.2.1): the drone's setpoint moves towards the
// waypoint by at most sp_rate_pos dt_ctrl (straight line) and sp_rate_yaw dt_ctrl (wrapped
// yaw difference) per control step, and the PID tracks the setpoint. A setpoint whose x is
// NaN is not set yet and starts at the drone's position and yaw. Reads and writes *spp.
__device__ __forceinline__ float4 dsl_setpoint(const Drone& d, const float4 wp, float4* spp, const DevConsts& c)
{
    float4 sp = *spp;
    if (isnan(sp.x)) {
        float roll, pitch, yaw;
        rpy_of(d.q, roll, pitch, yaw);
        sp = make_float4(d.p[0], d.p[1], d.p[2], yaw);
    }
    const float dx = wp.x - sp.x, dy = wp.y - sp.y, dz = wp.z - sp.z;
    const float n = sqrtf(dx * dx + dy * dy + dz * dz);
    const float s = n > c.sp_step_pos ? c.sp_step_pos / n : 1.f;
    sp.x += s * dx;
    sp.y += s * dy;
    sp.z += s * dz;
    float e = reduce_angle(wp.w) - sp.w;
    e -= 2.f * kPi * floorf((e + kPi) * (0.5f / kPi));
    e = fminf(c.sp_step_yaw, fmaxf(-c.sp_step_yaw, e));
    float y = sp.w + e;
    y -= 2.f * kPi * floorf((y + kPi) * (0.5f / kPi));
    sp.w = y;
    *spp = sp;
    return sp;
}

// Normalized RPM action (the tasks' [-1, 1] actions; the map is not printed). Reading: a
// clipped to [-1, 1], -1 -> 0, 0 -> HOVER_RPM, 1 -> MAX_RPM, linear on each side of hover.
__device__ __forceinline__ float normalized_rpm(float a, const DevConsts& c)
{
    a = fminf(1.f, fmaxf(-1.f, a));
    return a <= 0.f ? c.hover_rpm * (1.f + a) : c.hover_rpm + (c.max_rpm - c.hover_rpm) * a;
}

// The action types of Table "Action types" beyond RPM and PID, compiled into the
// runtime-flag kernels only:
//  RPM_NORM   four normalized values; ONE_D_RPM  act.x normalized, on all four motors;
//  VEL        body-frame [v_x, v_y, v_z, omega_z] through the PID: the position loop holds
//             the current position (zero error) with target velocity R v_body, the attitude
//             loop the current yaw with target body rate [0, 0, omega_z];
//  ATTITUDE   [T (N), roll*, pitch*, yaw rate] through the attitude loop (current yaw,
//             target body rate [0, 0, yaw rate]) and the mixer.
__device__ __forceinline__ void ext_action_rpm(Drone& d, const float4 act, int type, const DevConsts& c,
                                               float rpm[4])
{
    if (type == MDG_ACT_RPM_NORM) {
        rpm[0] = normalized_rpm(act.x, c);
        rpm[1] = normalized_rpm(act.y, c);
        rpm[2] = normalized_rpm(act.z, c);
        rpm[3] = normalized_rpm(act.w, c);
        return;
    }
    if (type == MDG_ACT_ONE_D_RPM) {
        const float r = normalized_rpm(act.x, c);
        rpm[0] = rpm[1] = rpm[2] = rpm[3] = r;
        return;
    }
    float roll, pitch, yaw;
    rpy_of(d.q, roll, pitch, yaw);
    float T = act.x, phi_t = act.y, theta_t = act.z;
    if (type == MDG_ACT_VEL) {
        const float qw = d.q[0], qx = d.q[1], qy = d.q[2], qz = d.q[3];
        const float vt[3] = {
            (1.f - 2.f * (qy * qy + qz * qz)) * act.x + 2.f * (qx * qy - qw * qz) * act.y + 2.f * (qx * qz + qw * qy) * act.z,
            2.f * (qx * qy + qw * qz) * act.x + (1.f - 2.f * (qx * qx + qz * qz)) * act.y + 2.f * (qy * qz - qw * qx) * act.z,
            2.f * (qx * qz - qw * qy) * act.x + 2.f * (qy * qz + qw * qx) * act.y + (1.f - 2.f * (qx * qx + qy * qy)) * act.z};
        float acc[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            d.ip[r] = fminf(c.pos_iclamp, fmaxf(-c.pos_iclamp, d.ip[r]));  // zero position error
            acc[r] = c.pos_ki[r] * d.ip[r] + c.pos_kd[r] * (vt[r] - d.v[r]);
        }
        acc[2] += c.g;
        T = c.mass * sqrt_approx(acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2]);
        float sps, cps;
        sincos_reduced(yaw, &sps, &cps);
        phi_t = (acc[0] * sps - acc[1] * cps) * c.inv_g;
        theta_t = (acc[0] * cps + acc[1] * sps) * c.inv_g;
    }
    float ye;
    attitude_and_mix<true>(d, T, phi_t, theta_t, yaw, act.w, roll, pitch, yaw, c, rpm, ye);
}

// Whether an action type runs the PID loops (and so reads and writes their integrals).
__device__ __forceinline__ bool uses_loops(int act)
{
    return act == MDG_ACT_PID || act == MDG_ACT_VEL || act == MDG_ACT_ATTITUDE;
}

// Downwash of Eq. downwash that drone j at p feels from one drone o of its environment:
// C1 (r_p/(4 dz))^2 exp(-dxy^2 / (2 beta^2)), beta = C2 dz + C3, when o is strictly above
// (dz > dz_min >= 0, which also excludes j itself) and dxy is within the lateral cut-off;
// otherwise 0. One reciprocal r = 1/(dz^2 beta^2) yields 1/dz^2 = beta^2 r and
// 1/beta^2 = dz^2 r; beta^2 is floored at 1e-12. Branch-free, so that unrolled pairs
// interleave; the select discards the values of excluded pairs. The reciprocal's argument
// is floored at 1e-30 so that those values stay finite (no inf * 0). For an included pair
// (beta^2 near 0.0121 at small dz) the floor binds only below dz ~ 1e-14 m, where the
// force is already ~1e27 N; there it stays at that value instead of growing as 1/dz^2.
__device__ __forceinline__ float downwash_pair(const float4 o, float px, float py, float pz, const DevConsts& c)
{
    const float dz = o.z - pz;
    const float dx = o.x - px, dy = o.y - py;
    const float d2 = dx * dx + dy * dy;
    const float beta = fmaf(c.dw_c2, dz, c.dw_c3);
    const float b2 = fmaxf(beta * beta, 1e-12f);
    const float dz2 = dz * dz;
    const float r = rcp_approx(fmaxf(dz2 * b2, 1e-30f));
    const float e = ex2_approx(-0.72134752044448170368f * d2 * dz2 * r);  // -0.5 log2(e)
    const float f = c.dw_k * b2 * r * e;
    return (dz > c.dw_dz_min && d2 < c.dw_max_xy2) ? f : 0.f;
}

// Downwash summed over the N drones of the environment in shared memory; jl is the
// drone's own index there. The loop is unrolled and branch-free so that independent pair
// terms interleave (a per-source warp vote that skips sources below the whole warp
// measured slower: its branch serialises the pairs). For a compile-time environment size
// that is a power of two up to 8 the loop visits the N - 1 other drones, (jl + i) mod N;
// otherwise it visits all N and the drone's own entry (dz = 0) drops out of the gate.
template <int kN>
__device__ __forceinline__ float downwash_sum(const float4* env_pos, int N_rt, int jl, float px, float py, float pz,
                                              const DevConsts& c)
{
    float acc = 0.f;
    if (kN > 0 && kN <= 8 && (kN & (kN - 1)) == 0) {
#pragma unroll
        for (int i = 1; i < (kN > 0 ? kN : 1); ++i) acc += downwash_pair(env_pos[(jl + i) & (kN - 1)], px, py, pz, c);
    } else if (kN > 0) {
#pragma unroll((kN > 0 && kN <= 8) ? kN : 8)
        for (int j = 0; j < kN; ++j) acc += downwash_pair(env_pos[j], px, py, pz, c);
    } else {
#pragma unroll 4
        for (int j = 0; j < N_rt; ++j) acc += downwash_pair(env_pos[j], px, py, pz, c);
    }
    return acc;
}

// Kernel variants beyond the compile-time physics subsets 0-7 (all take the physics flags
// at run time): 8 Euler substeps, kFlagsRK4 Runge-Kutta substeps, kFlagsGndRotor Euler
// substeps with Eq. ground at each rotor's height, kFlagsDR Euler substeps under domain
// randomization (with per-rotor heights too). The Runge-Kutta variants handle
// per-rotor heights too; variant 8 leaves that code out, so that its register allocation
// is the one the mixed-physics batches need.
constexpr int kFlagsRK4 = 9;
constexpr int kFlagsGndRotor = 10;
// Runge-Kutta variants with a compile-time physics subset s: kFlagsRK4Fixed + s.
constexpr int kFlagsRK4Fixed = 16;
__host__ __device__ constexpr bool rk4_variant(int f) { return f == kFlagsRK4 || f >= kFlagsRK4Fixed; }
// variants that take the physics flags (and the extra features) at run time
__host__ __device__ constexpr bool runtime_variant(int f) { return f >= 8 && f < kFlagsRK4Fixed; }
// the compile-time physics subset of a variant, or -1
__host__ __device__ constexpr int fixed_subset(int f) { return f < 8 ? f : (f >= kFlagsRK4Fixed ? f - kFlagsRK4Fixed : -1); }
constexpr int kFlagsDR = kVariantRandomized;  // Euler substeps with domain randomization, motor lag, latency, wind

// Eq. ground's increment along world +z, before its gate. With per-rotor heights rotor i
// is at height p_z + R20 x_i + R21 y_i, and its thrust f_i is recovered from T and the
// torques by the inverse mixing the PID uses (orthogonal rows).
template <int kFlags>
__device__ __forceinline__ float ground_increment(const Motor& m, float pz, float qw, float qx, float qy, float qz,
                                                  float R20, const DevConsts& c)
{
    if ((kFlags == kFlagsRK4 || kFlags == kFlagsGndRotor || kFlags == kFlagsDR) && c.gnd_rotor) {
        const float R21 = 2.f * (qy * qz + qw * qx);
        const float tx = c.alloc_xy * m.tau[0], ty = c.alloc_xy * m.tau[1], tz = c.alloc_z * m.tau[2];
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float f = 0.25f * (((m.T + c.mix_x[i] * tx) + c.mix_y[i] * ty) + ((i & 1) ? tz : -tz));
            const float h = fmaxf(fmaf(R20, c.rotor_x[i], fmaf(R21, c.rotor_y[i], pz)), c.h_clip);
            acc = fmaf(f, rcp_approx(h * h), acc);
        }
        return c.gnd_k * acc;
    }
    const float h = fmaxf(pz, c.h_clip);
    return c.gnd_k * m.T * rcp_approx(h * h);
}

// One substep: forces of Eq. motor/ground/drag/downwash, Newton-Euler, forward Euler
// and the exponential map, all from the start-of-substep state. `env_pos` points at the
// shared-memory positions of this drone's environment (N entries). kFlags (0..7) and kN
// (> 0) fix the physics subset and environment size at compile time for uniform batches;
// kFlags = 8 / kN <= 0 take them from the runtime arguments.
template <int kFlags, int kN>
__device__ __forceinline__ void substep(Drone& d, const Motor& m, int flags_rt, const float4* env_pos, int N_rt, int jl,
                                        const DevConsts& c, const float3 fe = float3{})
{
    const int flags = fixed_subset(kFlags) >= 0 ? fixed_subset(kFlags) : flags_rt;
    const float dt = c.dt_sim;
    // exponential map with the old body rate: q <- q (x) [cos(theta), sin(theta) w/|w|],
    // theta = |w| dt/2. sin(theta)/|w| = (dt/2) sinc(theta); for theta^2 <= 0.1 both factors
    // are the Taylor series of cos and sinc in theta^2 to theta^6 (truncation below 2.5e-9),
    // with neither a square root nor a division. Larger rotations per substep (|w| above
    // ~152 rad/s at 240 Hz) take sqrtf and the reduced sine/cosine (the rarely taken branch below).
    const float nw2 = d.w[0] * d.w[0] + d.w[1] * d.w[1] + d.w[2] * d.w[2];
    const float hdt = 0.5f * dt;
    const float t2 = nw2 * (hdt * hdt);
    float co = fmaf(t2, fmaf(t2, fmaf(t2, -1.3888889e-3f, 4.1666668e-2f), -0.5f), 1.0f);
    float k = hdt * fmaf(t2, fmaf(t2, fmaf(t2, -1.9841270e-4f, 8.3333333e-3f), -0.16666667f), 1.0f);

    // Only the body z axis in the world frame, r = R e_z (the third column of R), and R20 are
    // needed: thrust acts along r, the ground-effect gate reads R22 = r.z and R20, and the
    // drag of Eq. drag, R diag(c_xy, c_xy, c_z) R^T v, equals c_xy v + (c_z - c_xy)(r . v) r.
    const float qw = d.q[0], qx = d.q[1], qy = d.q[2], qz = d.q[3];
    const float r0 = 2.f * (qx * qz + qw * qy);
    const float r1 = 2.f * (qy * qz - qw * qx);
    const float r2 = 1.f - 2.f * (qx * qx + qy * qy);
    float F[3] = {r0 * m.T, r1 * m.T, r2 * m.T - c.mass * c.g};
    if (flags & MDG_GND) {
        // gate |roll| < pi/2 and |pitch| < pi/2: cos(roll) cos(pitch) = R22 > 0, |sin(pitch)| = |R20| < 1
        const float R20 = 2.f * (qx * qz - qw * qy);
        const float g = ground_increment<kFlags>(m, d.p[2], qw, qx, qy, qz, R20, c);
        F[2] += (r2 > 0.f && fabsf(R20) < 1.f) ? g : 0.f;
    }
    if (flags & MDG_DRAG) {
        const float rv = (r0 * d.v[0] + r1 * d.v[1]) + r2 * d.v[2];
        const float kxy = -m.wsum * c.c_xy, kr = -m.wsum * c.c_dz * rv;
        F[0] += kxy * d.v[0] + kr * r0;
        F[1] += kxy * d.v[1] + kr * r1;
        F[2] += kxy * d.v[2] + kr * r2;
    }
    if (flags & MDG_DW) F[2] -= downwash_sum<kN>(env_pos, N_rt, jl, d.p[0], d.p[1], d.p[2], c);
    if (kFlags == kFlagsDR) {  // the wind's force, world frame
        F[0] += fe.x;
        F[1] += fe.y;
        F[2] += fe.z;
    }
    // Newton-Euler: omega_dot = J^-1 (tau - omega x (J omega)), omega in the body frame
    const float Jw0 = c.J[0] * d.w[0], Jw1 = c.J[1] * d.w[1], Jw2 = c.J[2] * d.w[2];
    const float wd0 = c.inv_J[0] * (m.tau[0] - (d.w[1] * Jw2 - d.w[2] * Jw1));
    const float wd1 = c.inv_J[1] * (m.tau[1] - (d.w[2] * Jw0 - d.w[0] * Jw2));
    const float wd2 = c.inv_J[2] * (m.tau[2] - (d.w[0] * Jw1 - d.w[1] * Jw0));
    if (t2 > 0.1f) {
        // theta reduced by 2 pi, then the special function unit's sine and cosine (within
        // ~4e-7 absolute): no large-argument reduction code in the kernel
        const float nw = sqrtf(nw2);
        float sn;
        __sincosf(reduce_angle(hdt * nw), &sn, &co);
        k = sn / nw;
    }
    {
        const float bx = k * d.w[0], by = k * d.w[1], bz = k * d.w[2];
        const float nqw = qw * co - qx * bx - qy * by - qz * bz;
        const float nqx = qw * bx + qx * co + qy * bz - qz * by;
        const float nqy = qw * by - qx * bz + qy * co + qz * bx;
        const float nqz = qw * bz + qx * by - qy * bx + qz * co;
        const float inv = rsqrtf(nqw * nqw + nqx * nqx + nqy * nqy + nqz * nqz);
        d.q[0] = nqw * inv; d.q[1] = nqx * inv; d.q[2] = nqy * inv; d.q[3] = nqz * inv;
    }
    // forward Euler: p with the old v, v with the force of the old state
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        d.p[r] += dt * d.v[r];
        d.v[r] += dt * (F[r] * c.inv_mass);
    }
    d.w[0] += dt * wd0;
    d.w[1] += dt * wd1;
    d.w[2] += dt * wd2;
}

// x * 0 is a zero for finite x and NaN for an infinite or NaN x, so the sum of the
// products is zero exactly when the whole state is finite (one fused multiply-add each).
__device__ __forceinline__ bool finite_state(const Drone& d)
{
    float z = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) z = fmaf(d.w[r], 0.f, fmaf(d.v[r], 0.f, fmaf(d.p[r], 0.f, z)));
#pragma unroll
    for (int r = 0; r < 4; ++r) z = fmaf(d.q[r], 0.f, z);
    return z == 0.f;
}

// KIN observation [p, q, roll/pitch/yaw, v, w, a_prev] as five float4, given the angles.
__device__ __forceinline__ void kin_values(const Drone& d, const float a[4], const float rpy[3], float4 o[5])
{
    o[0] = make_float4(d.p[0], d.p[1], d.p[2], d.q[0]);
    o[1] = make_float4(d.q[1], d.q[2], d.q[3], rpy[0]);
    o[2] = make_float4(rpy[1], rpy[2], d.v[0], d.v[1]);
    o[3] = make_float4(d.v[2], d.w[0], d.w[1], d.w[2]);
    o[4] = make_float4(a[0], a[1], a[2], a[3]);
}

__device__ __forceinline__ void kin_values(const Drone& d, const float a[4], float4 o[5])
{
    float rpy[3];
    rpy_of(d.q, rpy[0], rpy[1], rpy[2]);
    kin_values(d, a, rpy, o);
}

// KIN row g; rpy: the angles when the caller has them (else computed here).
__device__ __forceinline__ void write_kin(float* __restrict__ kin, long long g, const Drone& d, const float a[4],
                                          const float* rpy = nullptr)
{
    float4 v[5];
    if (rpy) kin_values(d, a, rpy, v);
    else kin_values(d, a, v);
    float4* o = reinterpret_cast<float4*>(kin + 20 * g);
#pragma unroll
    for (int k = 0; k < 5; ++k) o[k] = v[k];
}

// The 4 nearest other drones of the environment (squared distance rounded in the
// order ((dx*dx + dy*dy) + dz*dz) without contraction, ties to the lower index), from the
// shared-memory positions of the environment; local indices, -1 where fewer exist.
// Candidates are taken in index order; each enters the last slot if strictly closer and
// moves up past strictly farther entries (branch-free selects), which keeps equal
// distances in index order.
template <int kN>
__device__ __forceinline__ void knn_best4(int j, const float p[3], const float4* env_pos, int N_rt, int bi[4])
{
    float b0 = INFINITY, b1 = INFINITY, b2 = INFINITY, b3 = INFINITY;
    int i0 = -1, i1 = -1, i2 = -1, i3 = -1;
    auto consider = [&](int k) {
        const float4 o = env_pos[k];
        const float dx = __fsub_rn(o.x, p[0]), dy = __fsub_rn(o.y, p[1]), dz = __fsub_rn(o.z, p[2]);
        float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        d2 = (k == j) ? INFINITY : d2;
        bool c = d2 < b3;
        b3 = c ? d2 : b3; i3 = c ? k : i3;
        c = b3 < b2;
        { const float tf = b2; const int ti = i2; b2 = c ? b3 : b2; i2 = c ? i3 : i2; b3 = c ? tf : b3; i3 = c ? ti : i3; }
        c = b2 < b1;
        { const float tf = b1; const int ti = i1; b1 = c ? b2 : b1; i1 = c ? i2 : i1; b2 = c ? tf : b2; i2 = c ? ti : i2; }
        c = b1 < b0;
        { const float tf = b0; const int ti = i0; b0 = c ? b1 : b0; i0 = c ? i1 : i0; b1 = c ? tf : b1; i1 = c ? ti : i1; }
    };
    if constexpr (kN == 4) {
        // The same list for four drones: the three others in index order, k = i + (i >= j),
        // sorted by the stable three-element network (0,1) (1,2) (0,1) that swaps only on a
        // strictly smaller distance; a distance that is not finite sorts last as +inf and
        // leaves its slot empty, as the insertion above would not take it.
        float dd[3];
        int kk[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int k = i + (i >= j ? 1 : 0);
            const float4 o = env_pos[k];
            const float dx = __fsub_rn(o.x, p[0]), dy = __fsub_rn(o.y, p[1]), dz = __fsub_rn(o.z, p[2]);
            const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            dd[i] = d2 < INFINITY ? d2 : INFINITY;
            kk[i] = k;
        }
        auto cx = [&](int u, int v) {
            const bool c = dd[v] < dd[u];
            const float tf = dd[u];
            const int ti = kk[u];
            dd[u] = c ? dd[v] : dd[u];
            kk[u] = c ? kk[v] : kk[u];
            dd[v] = c ? tf : dd[v];
            kk[v] = c ? ti : kk[v];
        };
        cx(0, 1);
        cx(1, 2);
        cx(0, 1);
#pragma unroll
        for (int i = 0; i < 3; ++i) bi[i] = dd[i] < INFINITY ? kk[i] : -1;
        bi[3] = -1;
        return;
    }
    if (kN > 0) {
#pragma unroll((kN > 0 && kN <= 8) ? kN : 4)
        for (int k = 0; k < kN; ++k) consider(k);
    } else {
        for (int k = 0; k < N_rt; ++k) consider(k);
    }
    bi[0] = i0; bi[1] = i1; bi[2] = i2; bi[3] = i3;
}

// Relative features [p_i - p_j, v_i - v_j] of the 4 slots (zeros for empty slots).
__device__ __forceinline__ void knn_features(const int bi[4], const Drone& d, const float4* env_pos,
                                             const float4* env_vel, float f[24])
{
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const bool ok = bi[s] >= 0;
        const float4 pp = env_pos[ok ? bi[s] : 0], vv = env_vel[ok ? bi[s] : 0];
        f[6 * s + 0] = ok ? pp.x - d.p[0] : 0.f;
        f[6 * s + 1] = ok ? pp.y - d.p[1] : 0.f;
        f[6 * s + 2] = ok ? pp.z - d.p[2] : 0.f;
        f[6 * s + 3] = ok ? vv.x - d.v[0] : 0.f;
        f[6 * s + 4] = ok ? vv.y - d.v[1] : 0.f;
        f[6 * s + 5] = ok ? vv.z - d.v[2] : 0.f;
    }
}

// Writes the neighbour observation of drone g: global indices and (optionally) features.
template <int kN>
__device__ __forceinline__ void write_knn(int4* __restrict__ nbr_idx, float* __restrict__ nbr_rel, long long g,
                                          long long env_first, int j, const Drone& d, const float4* env_pos,
                                          const float4* env_vel, int N_rt)
{
    int bi[4];
    knn_best4<kN>(j, d.p, env_pos, N_rt, bi);
    int4 idx;
    idx.x = bi[0] >= 0 ? (int)(env_first + bi[0]) : -1;
    idx.y = bi[1] >= 0 ? (int)(env_first + bi[1]) : -1;
    idx.z = bi[2] >= 0 ? (int)(env_first + bi[2]) : -1;
    idx.w = bi[3] >= 0 ? (int)(env_first + bi[3]) : -1;
    nbr_idx[g] = idx;
    if (nbr_rel) {
        float f[24];
        knn_features(bi, d, env_pos, env_vel, f);
        float4* o = reinterpret_cast<float4*>(nbr_rel + 24 * g);
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
    }
}

// Observations through per-warp staging: a lane's KIN (80 B) and feature (96 B) rows are
// strided 16-byte pieces, which the host link carries at a quarter of its rate and which
// reach L2 as half-written sectors. Each warp stages its 32 consecutive rows in shared
// memory (`stage`: 192 float4 of its own) and writes the contiguous span in 16-byte pieces,
// lane by lane. `g` is the lane's output row; the active lanes form a prefix of the warp
// and their rows are consecutive (lane 0's row + lane); every lane of the warp calls this.
template <int kN>
__device__ __forceinline__ void write_obs_staged(const StepArgs& a, float4* stage, bool active, long long g, int lane,
                                                 long long env_first, int j, const Drone& d, const float rpm[4],
                                                 const float4* env_pos, const float4* env_vel, int N_rt)
{
    const int n_act = __popc(__ballot_sync(0xffffffffu, active));
    const long long g0 = __shfl_sync(0xffffffffu, g, 0);
    if (active) {
        float4 v[5];
        kin_values(d, rpm, v);
#pragma unroll
        for (int k = 0; k < 5; ++k) stage[lane * 5 + k] = v[k];
    }
    __syncwarp();
    float4* kin = reinterpret_cast<float4*>(a.kin) + g0 * 5;
    for (int i = lane; i < n_act * 5; i += 32) kin[i] = stage[i];
    __syncwarp();
    if (active) {
        int bi[4];
        knn_best4<kN>(j, d.p, env_pos, N_rt, bi);
        int4 idx;
        idx.x = bi[0] >= 0 ? (int)(env_first + bi[0]) : -1;
        idx.y = bi[1] >= 0 ? (int)(env_first + bi[1]) : -1;
        idx.z = bi[2] >= 0 ? (int)(env_first + bi[2]) : -1;
        idx.w = bi[3] >= 0 ? (int)(env_first + bi[3]) : -1;
        a.nbr_idx[g] = idx;  // 16 bytes per lane, contiguous across the warp
        if (a.nbr_rel) {
            float f[24];
            knn_features(bi, d, env_pos, env_vel, f);
#pragma unroll
            for (int k = 0; k < 6; ++k) stage[lane * 6 + k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
        }
    }
    __syncwarp();
    if (a.nbr_rel) {
        float4* rel = reinterpret_cast<float4*>(a.nbr_rel) + g0 * 6;
        for (int i = lane; i < n_act * 6; i += 32) rel[i] = stage[i];
    }
}

// Shared-memory layout of the tile kernels (B = blockDim.x):
//   float4 pos[2][B] (double-buffered substep snapshot), float4 vel[B],
//   int off[B + 1] (tile-relative env offsets), int info[B] (flags | action type << 8)
__host__ __device__ constexpr size_t tile_smem_bytes(int B) { return (size_t)B * 48 + (size_t)(2 * B + 1) * 4; }
// ... followed, for observations to host memory, by 192 float4 of staging per warp
__host__ __device__ constexpr size_t obs_stage_offset(int B) { return (tile_smem_bytes(B) + 15) / 16 * 16; }
__host__ __device__ constexpr size_t obs_stage_bytes(int B) { return (size_t)(B / 32) * 192 * 16; }

// The block's tile: whole environments, given by the host's tile table, or computed
// arithmetically when every environment has the same size (uniform batches).
struct TileInfo {
    long long first_drone;
    int n_drones, first_env, n_envs, bits;
};

// This thread's environment: first drone (tile-local), size, flags and action type.
struct EnvSlot {
    int ls, N, flags, act;
    int id;  // global environment index
};

__device__ __forceinline__ TileInfo get_tile(const StepArgs& a)
{
    TileInfo ti;
    if (a.uniform_N > 0) {
        ti.first_env = blockIdx.x * a.envs_per_tile;
        ti.n_envs = min(a.envs_per_tile, a.n_envs - ti.first_env);
        ti.first_drone = (long long)ti.first_env * a.uniform_N;
        ti.n_drones = ti.n_envs * a.uniform_N;
        ti.bits = a.uniform_bits;
    } else {
        const Tile t = a.tiles[blockIdx.x];
        ti.first_drone = t.x;
        ti.n_drones = t.y;
        ti.first_env = t.z;
        ti.n_envs = t.w & kTileEnvMask;
        ti.bits = t.w & ~kTileEnvMask;
    }
    // debug builds: the tile lies inside the batch, fits the block and covers whole environments
    if (!MDG_CHECK(ti.first_drone >= 0 && ti.n_drones >= 0 && ti.n_drones <= (int)blockDim.x &&
                       ti.first_drone + ti.n_drones <= a.n && ti.first_env >= 0 && ti.n_envs >= 0 &&
                       ti.first_env + ti.n_envs <= a.n_envs &&
                       (a.uniform_N > 0 || (a.env_off[ti.first_env] == ti.first_drone &&
                                            a.env_off[ti.first_env + ti.n_envs] == ti.first_drone + ti.n_drones)),
                   a.status)) {
        ti.n_drones = 0;
        ti.n_envs = 0;
    }
    return ti;
}

// debug builds: a thread's environment contains the thread and lies inside the tile
__device__ __forceinline__ void check_env(EnvSlot& e, int t, int n_drones, uint32_t* status)
{
    if (t < n_drones && !MDG_CHECK(e.ls >= 0 && e.N >= 1 && e.ls <= t && t < e.ls + e.N && e.ls + e.N <= n_drones, status)) {
        e.ls = 0;
        e.N = 0;
    }
}


// kN > 0: the batch is uniform with kN drones per environment (the compile-time variants
// are launched only then), so the division below is by a constant.
template <int kN = 0>
__device__ __forceinline__ EnvSlot tile_env(const StepArgs& a, const TileInfo& ti, int* s_off, int* s_info)
{
    const int t = threadIdx.x;
    EnvSlot e = {0, 0, 0, 0, 0};
    if (a.uniform_N > 0) {
        if (t < ti.n_drones) {
            const int k = t / (kN > 0 ? kN : a.uniform_N);
            e.id = ti.first_env + k;
            e.ls = k * a.uniform_N;
            e.N = a.uniform_N;
            e.flags = a.env_flags[ti.first_env + k];
            e.act = a.act_type == MDG_ACT_MIXED ? (int)a.env_act[ti.first_env + k] : a.act_type;
        }
        check_env(e, t, ti.n_drones, a.status);
        return e;
    }
    const int B = blockDim.x;
    for (int i = t; i <= ti.n_envs; i += B) s_off[i] = a.env_off[ti.first_env + i] - (int)ti.first_drone;
    for (int i = t; i < ti.n_envs; i += B) {
        const int act = a.act_type == MDG_ACT_MIXED ? (int)a.env_act[ti.first_env + i] : a.act_type;
        s_info[i] = (int)a.env_flags[ti.first_env + i] | (act << 8);
    }
    __syncthreads();
    if (t < ti.n_drones) {
        int lo = 0, hi = ti.n_envs - 1;  // largest env with s_off[env] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        e.ls = s_off[lo];
        e.N = s_off[lo + 1] - e.ls;
        e.flags = s_info[lo] & 0xff;
        e.act = s_info[lo] >> 8;
        e.id = ti.first_env + lo;
    }
    check_env(e, t, ti.n_drones, a.status);
    return e;
}

// ---- domain randomization, motor lag, action latency and wind (kFlags == kFlagsDR) ----

constexpr unsigned long long kStreamWind = 21;  // random stream of the wind draws

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014): the output function of its counter-based form.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// U[0, 1) with 24 random bits (exact in float) for the counters (seed, stream, step,
// index, comp), each mixed in by one SplitMix64 round. The rounds of (seed, stream, step,
// index) form a prefix that all components of one draw share: counter_prefix mixes it once
// and prefix_uniform adds the component's round (the same values as mixing all five).
__device__ __forceinline__ unsigned long long counter_prefix(unsigned long long seed, unsigned long long stream,
                                                             unsigned long long step, unsigned long long index)
{
    unsigned long long h = splitmix64(seed);
    h = splitmix64(h ^ stream);
    h = splitmix64(h ^ step);
    return splitmix64(h ^ index);
}

__device__ __forceinline__ float prefix_uniform(unsigned long long prefix, unsigned long long comp)
{
    return (float)(splitmix64(prefix ^ comp) >> 40) * (1.f / 16777216.f);
}

// The physics constants of an environment under its randomization row: factors on mass,
// inertia, arm, k_f, k_m, c_xy, c_z, C_gnd, C1 and g (the controller keeps c).
__device__ __forceinline__ DevConsts randomized_consts(const DevConsts& c, const float* row)
{
    DevConsts p = c;
    const float fm = row[MDG_DR_MASS];
    p.mass = c.mass * fm;
    p.inv_mass = c.inv_mass / fm;
    p.g = c.g * row[MDG_DR_G];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        p.J[r] = c.J[r] * row[MDG_DR_J + r];
        p.inv_J[r] = c.inv_J[r] / row[MDG_DR_J + r];
    }
    const float fl = row[MDG_DR_ARM], fkf = row[MDG_DR_KF], fkm = row[MDG_DR_KM];
    p.l_sqrt2 = c.l_sqrt2 * fl;
    p.alloc_xy = c.alloc_xy / fl;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        p.rotor_x[i] = c.rotor_x[i] * fl;
        p.rotor_y[i] = c.rotor_y[i] * fl;
    }
    p.kf = c.kf * fkf;
    p.km = c.km * fkm;
    p.alloc_z = c.alloc_z * (fkf / fkm);
    p.c_xy = c.c_xy * row[MDG_DR_CXY];
    p.c_z = c.c_z * row[MDG_DR_CZ];
    p.c_dz = p.c_z - p.c_xy;
    p.gnd_k = c.gnd_k * row[MDG_DR_CGND];
    p.dw_k = c.dw_k * row[MDG_DR_C1];
    return p;
}

// Action latency: the action received enters the drone's shift register and the one
// received `delay` control steps ago comes out (an empty register is first filled with
// the action received).
__device__ __forceinline__ float4 delayed_action(const StepArgs& a, long long g, const float4 act, int delay)
{
    float4* h = a.rand->hist + g;
    const int depth = a.rand->depth;
    if (isnan(h[0].x)) {
        for (int k = 0; k < depth; ++k) h[k * a.n] = act;
        return act;
    }
    float4 out = act;
    for (int k = depth - 1; k > 0; --k) {
        const float4 v = h[(k - 1) * a.n];
        h[k * a.n] = v;
        if (k == delay) out = v;
    }
    h[0] = act;
    return out;
}

// One control step of an environment's wind (Section 3.5): advances its state s0 = (Dryden
// x, gust phase s or -1), s1 = (gust direction, steps taken) and returns the direct force
// (gusts, sinusoid) and the wind velocity the quadratic drag sees (steady wind, Dryden).
// CONSTANT: the steady wind; DRYDEN: x <- alpha x + sigma sqrt(1 - alpha^2) xi per component,
// alpha = exp(-dt V / L), L = h / (0.177 + 8.23e-4 h)^1.2, xi by Box-Muller; GUST: an idle
// field starts a gust with the set probability, direction uniform on the sphere, force
// A sin(pi s) while its phase s <= 1; SINUSOIDAL: A [sin wt, cos wt, 0.3 sin 2wt]. The gust
// phase decides when a gust ends and advances in single precision.
__device__ __forceinline__ void wind_step(const float* row, float4& s0, float4& s1, unsigned long long seed, int env,
                                          float dt, float F[3], float vw[3])
{
    const int model = (int)row[MDG_DR_WIND];
    const unsigned long long step = (unsigned long long)s1.w;
    const unsigned long long wind_key = counter_prefix(seed, kStreamWind, step, env);
    F[0] = F[1] = F[2] = vw[0] = vw[1] = vw[2] = 0.f;
    if (model & MDG_WIND_CONSTANT) {
        vw[0] += row[MDG_DR_VWIND];
        vw[1] += row[MDG_DR_VWIND + 1];
        vw[2] += row[MDG_DR_VWIND + 2];
    }
    if (model & MDG_WIND_DRYDEN) {
        const float h = row[MDG_DR_DRY_H];
        const float L = h / powf(0.177f + 8.23e-4f * h, 1.2f);
        const float alpha = expf(-dt * row[MDG_DR_DRY_V] / L);
        const float u1 = 1.f - prefix_uniform(wind_key, 0);
        const float u2 = prefix_uniform(wind_key, 1);
        const float u3 = 1.f - prefix_uniform(wind_key, 2);
        const float u4 = prefix_uniform(wind_key, 3);
        const float r1 = sqrtf(-2.f * logf(u1)), r2 = sqrtf(-2.f * logf(u3));
        float s2, c2, s4, c4;
        // sin and cos of 2 pi u as sincospif(2 u): exact argument reduction, and without the
        // large-argument path a general sincosf inlines at every call
        sincospif(2.f * u2, &s2, &c2);
        sincospif(2.f * u4, &s4, &c4);
        const float sc = row[MDG_DR_DRY_SIGMA] * sqrtf(fmaxf(0.f, 1.f - alpha * alpha));
        s0.x = alpha * s0.x + sc * (r1 * c2);
        s0.y = alpha * s0.y + sc * (r1 * s2);
        s0.z = alpha * s0.z + sc * (r2 * c4);
        vw[0] += s0.x;
        vw[1] += s0.y;
        vw[2] += s0.z;
    }
    if (model & MDG_WIND_GUST) {
        if (s0.w < 0.f && prefix_uniform(wind_key, 4) < row[MDG_DR_GUST_P]) {
            const float z = 2.f * prefix_uniform(wind_key, 5) - 1.f;
            const float u6 = prefix_uniform(wind_key, 6);  // direction angle 2 pi u6
            const float rho = sqrtf(fmaxf(0.f, 1.f - z * z));
            float sn, cs;
            sincospif(2.f * u6, &sn, &cs);
            s0.w = 0.f;
            s1.x = rho * cs;
            s1.y = rho * sn;
            s1.z = z;
        }
        if (s0.w >= 0.f) {
            const float amp = row[MDG_DR_GUST_A] * sinpif(s0.w);
            F[0] += amp * s1.x;
            F[1] += amp * s1.y;
            F[2] += amp * s1.z;
            s0.w += dt / row[MDG_DR_GUST_T];
            if (s0.w > 1.f) s0.w = -1.f;
        }
    }
    if (model & MDG_WIND_SINUSOIDAL) {
        const float wt = row[MDG_DR_SIN_W] * ((float)step * dt), A = row[MDG_DR_SIN_A];
        F[0] += A * sinf(wt);
        F[1] += A * cosf(wt);
        F[2] += A * 0.3f * sinf(2.f * wt);
    }
    s1.w = (float)(step + 1);
}

constexpr unsigned long long kStreamObs = 22;  // random stream of the observation noise

// The KIN observation of d (RPMs a4) with the row's sensor noise: Gaussian (Box-Muller on the
// counters (seed, kStreamObs, step, drone, 0..11)) of the row's sigmas on the position (0-2),
// roll/pitch/yaw (3-5), velocity (6-8) and body rate (9-11), plus the drone's sticky
// per-episode bias on the same channels when obs_bias ([n][12] as three float4) is given;
// stored at kin_row[0..19].
__device__ __forceinline__ void noisy_kin(float* kin_row, const Drone& d, const float a4[4], const float* row,
                                          unsigned long long seed, unsigned long long step, long long g,
                                          const float4* obs_bias)
{
    float4 v[5];
    kin_values(d, a4, v);
    const float sp = row[MDG_DR_NOISE_P], sv = row[MDG_DR_NOISE_V], sr = row[MDG_DR_NOISE_RPY],
                sw = row[MDG_DR_NOISE_W];
    if (sp > 0.f || sv > 0.f || sr > 0.f || sw > 0.f) {
        float xi[12];
        const unsigned long long key = counter_prefix(seed, kStreamObs, step, g);
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const float u1 = 1.f - prefix_uniform(key, 2 * m);
            const float u2 = prefix_uniform(key, 2 * m + 1);
            const float r = sqrtf(-2.f * logf(u1));
            float sn, cs;
            sincospif(2.f * u2, &sn, &cs);  // sin and cos of 2 pi u2
            xi[2 * m] = r * cs;
            xi[2 * m + 1] = r * sn;
        }
        v[0].x += sp * xi[0];
        v[0].y += sp * xi[1];
        v[0].z += sp * xi[2];
        v[1].w += sr * xi[3];
        v[2].x += sr * xi[4];
        v[2].y += sr * xi[5];
        v[2].z += sv * xi[6];
        v[2].w += sv * xi[7];
        v[3].x += sv * xi[8];
        v[3].y += sw * xi[9];
        v[3].z += sw * xi[10];
        v[3].w += sw * xi[11];
    }
    if (obs_bias) {  // [p (3), rpy (3), v (3), w (3)] as (p.xyz, roll) (pitch, yaw, v.xy) (v.z, w.xyz)
        const float4 b0 = obs_bias[3 * g], b1 = obs_bias[3 * g + 1], b2 = obs_bias[3 * g + 2];
        v[0].x += b0.x;
        v[0].y += b0.y;
        v[0].z += b0.z;
        v[1].w += b0.w;
        v[2].x += b1.x;
        v[2].y += b1.y;
        v[2].z += b1.z;
        v[2].w += b1.w;
        v[3].x += b2.x;
        v[3].y += b2.y;
        v[3].z += b2.z;
        v[3].w += b2.w;
    }
    float4* o = reinterpret_cast<float4*>(kin_row);
#pragma unroll
    for (int k = 0; k < 5; ++k) o[k] = v[k];
}

constexpr unsigned long long kStreamInit = 23;  // random stream of the per-episode initial states
constexpr unsigned long long kStreamBias = 24;  // random stream of the per-episode observation bias

// Episode reset (Section 3.5: the "init" row of Table "Recommended domain-randomization
// ranges" and the sticky per-episode observation bias of its recommendation (iii)), one thread
// per drone g: uniforms u_k = U(seed, kStreamInit, episode, g, k),
//   p0 = nominal.xyz + r_p (2 u_0..2 - 1), (roll, pitch, yaw)0 = (0, 0, nominal.w) + r_a (2 u_3..5 - 1),
//   q0 = the quaternion of Rz(yaw) Ry(pitch) Rx(roll), v0 = r_v (2 u_6..8 - 1), w0 = 0,
// integrals and the last RPMs zero; with a bias buffer, b_k = sigma[k / 3] xi_k by Box-Muller on
// U(seed, kStreamBias, episode, g, 2m) and (.., 2m + 1), k = 0..11.
__global__ void __launch_bounds__(256) reset_kernel(const ResetArgs r)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= r.n) return;
    const unsigned long long key = counter_prefix(r.seed, kStreamInit, r.episode, (unsigned long long)g);
    float u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = 2.f * prefix_uniform(key, k) - 1.f;
    const float4 nom = r.nominal[g];
    const float roll = r.range_att * u[3], pitch = r.range_att * u[4], yaw = nom.w + r.range_att * u[5];
    float sr, cr, sp, cp, sy, cy;  // of the half angles (once per episode: the accurate sincosf)
    sincosf(0.5f * roll, &sr, &cr);
    sincosf(0.5f * pitch, &sp, &cp);
    sincosf(0.5f * yaw, &sy, &cy);
    const float qw = cr * cp * cy + sr * sp * sy;
    const float qx = sr * cp * cy - cr * sp * sy;
    const float qy = cr * sp * cy + sr * cp * sy;
    const float qz = cr * cp * sy - sr * sp * cy;
    const float px = nom.x + r.range_pos * u[0], py = nom.y + r.range_pos * u[1], pz = nom.z + r.range_pos * u[2];
    const float vx = r.range_vel * u[6], vy = r.range_vel * u[7], vz = r.range_vel * u[8];
    float4* S = r.state;
    S[g] = make_float4(px, py, pz, qw);
    S[r.n + g] = make_float4(qx, qy, qz, vx);
    S[2 * r.n + g] = make_float4(vy, vz, 0.f, 0.f);
    S[3 * r.n + g] = make_float4(0.f, 0.f, 0.f, 0.f);
    S[4 * r.n + g] = make_float4(0.f, 0.f, 0.f, 0.f);
    S[5 * r.n + g] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r.obs_bias) {
        const unsigned long long bkey = counter_prefix(r.seed, kStreamBias, r.episode, (unsigned long long)g);
        float b[12];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const float u1 = 1.f - prefix_uniform(bkey, 2 * m);
            const float u2 = prefix_uniform(bkey, 2 * m + 1);
            const float rho = sqrtf(-2.f * logf(u1));
            float sn, cs;
            sincospif(2.f * u2, &sn, &cs);  // sin and cos of 2 pi u2
            b[2 * m] = r.sigma[(2 * m) / 3] * rho * cs;
            b[2 * m + 1] = r.sigma[(2 * m + 1) / 3] * rho * sn;
        }
        float4* o = r.obs_bias + 3 * g;
        o[0] = make_float4(b[0], b[1], b[2], b[3]);
        o[1] = make_float4(b[4], b[5], b[6], b[7]);
        o[2] = make_float4(b[8], b[9], b[10], b[11]);
    }
}

// The substeps of one control step under randomization, called by every thread of the
// block (barriers inside). From the step's start: the environment's wind (each drone
// evaluates it, the environment's first drone stores the new state once the block has read
// the old one) and the drone's drag from it, held over the substeps; the randomized
// constants; each motor's command (its RPM times its bias, saturated at MAX_RPM times the
// factor). Before each substep every rotor speed relaxes towards its command,
// n <- c + (n - c) exp(-dt/tau) (exact for a first-order lag under a constant command).
// Observations (when kin_row is given): with a sensor delay the noisy KIN of the step's
// start (the state d and the RPMs a_pre of that moment) is written here, and `delayed`
// tells the caller not to write the end-of-step one; `step` returns the wind step counter
// of this control step (the noise's key).
template <int kN>
__device__ __forceinline__ void randomized_substeps(const StepArgs& a, Drone& d, const float rpm[4], const EnvSlot& env,
                                                    float4* s_pos, int B, int t, long long g, bool active,
                                                    bool tile_dw, bool warp_local, int& ph, float* kin_row,
                                                    const float a_pre[4], bool& delayed, unsigned long long& step)
{
    const RandArgs& R = *a.rand;
    const float* row = R.dr + (long long)env.id * MDG_DR_PARAMS;
    __syncthreads();  // the previous control step's wind state is stored
    float4 s0 = {}, s1 = {}, ms = {};
    float cmd[4] = {0.f, 0.f, 0.f, 0.f}, lag = 0.f;
    float3 fe = {};
    DevConsts pc = a.c;
    delayed = false;
    step = 0;
    if (active) {
        s0 = R.wind[2LL * env.id];
        s1 = R.wind[2LL * env.id + 1];
        step = (unsigned long long)s1.w;
        delayed = row[MDG_DR_OBS_DELAY] == 1.f;
        if (kin_row && delayed) noisy_kin(kin_row, d, a_pre, row, R.seed, step, g, R.obs_bias);
        float Fd[3], vw[3];
        wind_step(row, s0, s1, R.seed, env.id, a.c.dt_ctrl, Fd, vw);
        const int model = (int)row[MDG_DR_WIND];
        if (model & (MDG_WIND_CONSTANT | MDG_WIND_DRYDEN)) {
            const float vr[3] = {vw[0] - d.v[0], vw[1] - d.v[1], vw[2] - d.v[2]};
            const float k = row[MDG_DR_KDRAG] * sqrtf(vr[0] * vr[0] + vr[1] * vr[1] + vr[2] * vr[2]);
            Fd[0] += k * vr[0];
            Fd[1] += k * vr[1];
            Fd[2] += k * vr[2];
        }
        fe = make_float3(Fd[0], Fd[1], Fd[2]);
        pc = randomized_consts(a.c, row);
        const float sat = a.c.max_rpm * row[MDG_DR_MAXRPM];
#pragma unroll
        for (int i = 0; i < 4; ++i) cmd[i] = fminf(rpm[i] * row[MDG_DR_BIAS + i], sat);
        const float tau = row[MDG_DR_TAU];
        lag = tau > 0.f ? expf(-a.c.dt_sim / tau) : 0.f;
        ms = R.motor[g];
        if (isnan(ms.x)) ms.x = cmd[0];
        if (isnan(ms.y)) ms.y = cmd[1];
        if (isnan(ms.z)) ms.z = cmd[2];
        if (isnan(ms.w)) ms.w = cmd[3];
    }
    __syncthreads();  // every drone has read the wind state
    if (active && t == env.ls) {
        R.wind[2LL * env.id] = s0;
        R.wind[2LL * env.id + 1] = s1;
    }
    for (int s = 0; s < a.n_sub; ++s, ++ph) {
        float4* buf = s_pos + (ph & 1) * B;
        if (tile_dw) {
            buf[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
            if (warp_local) __syncwarp();
            else __syncthreads();
        }
        if (active) {
            ms.x = cmd[0] + (ms.x - cmd[0]) * lag;
            ms.y = cmd[1] + (ms.y - cmd[1]) * lag;
            ms.z = cmd[2] + (ms.z - cmd[2]) * lag;
            ms.w = cmd[3] + (ms.w - cmd[3]) * lag;
            const float n[4] = {ms.x, ms.y, ms.z, ms.w};
            substep<kFlagsDR, kN>(d, motor(n, pc), env.flags, buf + env.ls, env.N, t - env.ls, pc, fe);
        }
    }
    if (active) R.motor[g] = ms;
}

// ---- fourth-order Runge-Kutta substeps (MDG_INTEGRATOR_RK4) ----

// Time derivative of one drone's state at a Runge-Kutta stage: the forces of Eq. motor,
// ground, drag and downwash at the stage state s (its quaternion taken at unit length for
// the forces; env_pos holds the environment's stage positions) and Newton-Euler:
// p' = v, q' = 1/2 q (x) [0, w] (body rate on the right), v' = F/m,
// w' = J^-1 (tau - w x (J w)). The force expressions are those of substep().
struct StateRate {
    float p[3], q[4], v[3], w[3];
};

template <int kFlags, int kN>
__device__ __forceinline__ void stage_rate(const Drone& s, const Motor& m, int flags_rt, const float4* env_pos,
                                           int N_rt, int jl, const DevConsts& c, StateRate& k)
{
    const int flags = fixed_subset(kFlags) >= 0 ? fixed_subset(kFlags) : flags_rt;
    const float qi = rsqrtf(s.q[0] * s.q[0] + s.q[1] * s.q[1] + s.q[2] * s.q[2] + s.q[3] * s.q[3]);
    const float qw = s.q[0] * qi, qx = s.q[1] * qi, qy = s.q[2] * qi, qz = s.q[3] * qi;
    const float r0 = 2.f * (qx * qz + qw * qy);
    const float r1 = 2.f * (qy * qz - qw * qx);
    const float r2 = 1.f - 2.f * (qx * qx + qy * qy);
    float F[3] = {r0 * m.T, r1 * m.T, r2 * m.T - c.mass * c.g};
    if (flags & MDG_GND) {
        const float R20 = 2.f * (qx * qz - qw * qy);
        const float g = ground_increment<kFlags>(m, s.p[2], qw, qx, qy, qz, R20, c);
        F[2] += (r2 > 0.f && fabsf(R20) < 1.f) ? g : 0.f;
    }
    if (flags & MDG_DRAG) {
        const float rv = (r0 * s.v[0] + r1 * s.v[1]) + r2 * s.v[2];
        const float kxy = -m.wsum * c.c_xy, kr = -m.wsum * c.c_dz * rv;
        F[0] += kxy * s.v[0] + kr * r0;
        F[1] += kxy * s.v[1] + kr * r1;
        F[2] += kxy * s.v[2] + kr * r2;
    }
    if (flags & MDG_DW) F[2] -= downwash_sum<kN>(env_pos, N_rt, jl, s.p[0], s.p[1], s.p[2], c);
    const float Jw0 = c.J[0] * s.w[0], Jw1 = c.J[1] * s.w[1], Jw2 = c.J[2] * s.w[2];
    k.w[0] = c.inv_J[0] * (m.tau[0] - (s.w[1] * Jw2 - s.w[2] * Jw1));
    k.w[1] = c.inv_J[1] * (m.tau[1] - (s.w[2] * Jw0 - s.w[0] * Jw2));
    k.w[2] = c.inv_J[2] * (m.tau[2] - (s.w[0] * Jw1 - s.w[1] * Jw0));
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        k.p[r] = s.v[r];
        k.v[r] = F[r] * c.inv_mass;
    }
    // 1/2 q (x) [0, w] with the stage quaternion as it is
    k.q[0] = 0.5f * (-s.q[1] * s.w[0] - s.q[2] * s.w[1] - s.q[3] * s.w[2]);
    k.q[1] = 0.5f * (s.q[0] * s.w[0] + s.q[2] * s.w[2] - s.q[3] * s.w[1]);
    k.q[2] = 0.5f * (s.q[0] * s.w[1] - s.q[1] * s.w[2] + s.q[3] * s.w[0]);
    k.q[3] = 0.5f * (s.q[0] * s.w[2] + s.q[1] * s.w[1] - s.q[2] * s.w[0]);
}

// n_sub Runge-Kutta substeps of every drone of the block: k1 = f(x), k2 = f(x + dt/2 k1),
// k3 = f(x + dt/2 k2), k4 = f(x + dt k3), x+ = x + dt/6 (k1 + 2 k2 + 2 k3 + k4), q
// renormalised. Each stage publishes its positions into the double-buffered shared array
// (`ph` counts the publications, so that consecutive stages alternate buffers) and every
// drone of the environment evaluates the downwash at that stage's positions. Called by
// every thread of the block (barriers inside).
template <int kFlags, int kN>
__device__ __forceinline__ void rk4_substeps(Drone& d, const Motor& m, const EnvSlot& env, float4* s_pos, int B,
                                             int t, bool active, bool tile_dw, bool warp_local, int n_sub, int& ph,
                                             const DevConsts& c)
{
    const float dt = c.dt_sim;
    for (int s = 0; s < n_sub; ++s) {
        Drone st = d;
        StateRate sum = {};
#pragma unroll 1
        for (int stage = 0; stage < 4; ++stage, ++ph) {
            float4* buf = s_pos + (ph & 1) * B;
            if (tile_dw) {
                buf[t] = make_float4(st.p[0], st.p[1], st.p[2], 0.f);
                if (warp_local) __syncwarp();
                else __syncthreads();
            }
            if (active) {
                StateRate k;
                stage_rate<kFlags, kN>(st, m, env.flags, buf + env.ls, env.N, t - env.ls, c, k);
                const float wgt = (stage == 0 || stage == 3) ? 1.f : 2.f;
                const float h = stage < 2 ? 0.5f * dt : dt;  // offset of the next stage
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    sum.p[r] += wgt * k.p[r];
                    sum.v[r] += wgt * k.v[r];
                    sum.w[r] += wgt * k.w[r];
                    st.p[r] = d.p[r] + h * k.p[r];
                    st.v[r] = d.v[r] + h * k.v[r];
                    st.w[r] = d.w[r] + h * k.w[r];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    sum.q[r] += wgt * k.q[r];
                    st.q[r] = d.q[r] + h * k.q[r];
                }
            }
        }
        if (active) {
            const float h6 = dt * (1.f / 6.f);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                d.p[r] += h6 * sum.p[r];
                d.v[r] += h6 * sum.v[r];
                d.w[r] += h6 * sum.w[r];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) d.q[r] += h6 * sum.q[r];
            const float inv = rsqrtf(d.q[0] * d.q[0] + d.q[1] * d.q[1] + d.q[2] * d.q[2] + d.q[3] * d.q[3]);
#pragma unroll
            for (int r = 0; r < 4; ++r) d.q[r] *= inv;
        }
    }
}

// Variants with a compile-time environment size (kN > 0), and the runtime-size variant
// kN = -1, run blocks of at most kSmallBlock threads and may use up to 128 registers;
// the kN = 0 variant takes any block size (64 registers).
constexpr int kSmallBlock = 256;
template <int kN>
struct StepBounds {
    static constexpr int threads = kN != 0 ? kSmallBlock : 1024;
    static constexpr int min_blocks = kN != 0 ? 2 : 1;
};

template <bool kObs, int kFlags, int kN>
__global__ void __launch_bounds__(StepBounds<kN>::threads, StepBounds<kN>::min_blocks) step_kernel(const StepArgs a)
{
    extern __shared__ float4 smem[];
    const int B = blockDim.x;
    float4* s_pos = smem;          // [2][B]
    float4* s_vel = smem + 2 * B;  // [B]
    int* s_off = reinterpret_cast<int*>(smem + 3 * B);
    int* s_info = s_off + B + 1;

    const TileInfo tile = get_tile(a);
    const int t = threadIdx.x;
    const bool active = t < tile.n_drones;
    const long long g = tile.first_drone + t;
    // Issue the state and action loads before the environment lookup so that their
    // latency overlaps it.
    float4 s0 = {}, s1 = {}, s2 = {}, s3 = {}, s4 = {}, act = {};
    if (active) {
        s0 = a.state[g];
        s1 = a.state[a.n + g];
        s2 = a.state[2 * a.n + g];
        s3 = a.state[3 * a.n + g];
        if (a.act_type != MDG_ACT_RPM) s4 = a.state[4 * a.n + g];
        act = a.action[g];
    }
    const EnvSlot env = tile_env<kN>(a, tile, s_off, s_info);
    const bool is_pid = env.act == MDG_ACT_PID;
    const bool loops = is_pid || (runtime_variant(kFlags) && uses_loops(env.act));

    Drone d;
    unpack_state(s0, s1, s2, s3, s4, d);
    float rpm[4] = {0.f, 0.f, 0.f, 0.f};
    float a_pre[4] = {0.f, 0.f, 0.f, 0.f};  // randomization: the RPMs of the step's start (delayed observations)
    bool delayed = false;
    unsigned long long obs_step = 0;
    if (active) {
        if constexpr (kFlags == kFlagsDR) {  // action latency
            act = delayed_action(a, g, act, (int)a.rand->dr[(long long)env.id * MDG_DR_PARAMS + MDG_DR_DELAY]);
            if (kObs) {
                const float4 p5 = a.state[5 * a.n + g];
                a_pre[0] = p5.x, a_pre[1] = p5.y, a_pre[2] = p5.z, a_pre[3] = p5.w;
            }
        }
        if (runtime_variant(kFlags) && env.act >= MDG_ACT_RPM_NORM) {
            ext_action_rpm(d, act, env.act, a.c, rpm);
        } else if (is_pid) {
            float ep[3], ye;
            const float4 wp = (runtime_variant(kFlags) && a.c.dsl) ? dsl_setpoint(d, act, a.setpoints + g, a.c) : act;
            pid(d, wp, a.c, rpm, ep, ye);
        } else {
            rpm[0] = fminf(a.c.max_rpm, fmaxf(0.f, act.x));
            rpm[1] = fminf(a.c.max_rpm, fmaxf(0.f, act.y));
            rpm[2] = fminf(a.c.max_rpm, fmaxf(0.f, act.z));
            rpm[3] = fminf(a.c.max_rpm, fmaxf(0.f, act.w));
        }
    }
    const Motor m = motor(rpm, a.c);
    // Downwash needs the start-of-substep positions of the environment: published in a
    // double-buffered shared array, one barrier per substep (a warp barrier when every
    // environment of the tile lies inside one warp).
    const bool tile_dw = (tile.bits & kTileAnyDW) != 0;
    const bool warp_local = (tile.bits & kTileWarpLocal) != 0;
    int ph = 0;  // position publications (the double buffer's parity)
    if constexpr (rk4_variant(kFlags)) {
        rk4_substeps<kFlags, kN>(d, m, env, s_pos, B, t, active, tile_dw, warp_local, a.n_sub, ph, a.c);
    } else if constexpr (kFlags == kFlagsDR) {
        randomized_substeps<kN>(a, d, rpm, env, s_pos, B, t, g, active, tile_dw, warp_local, ph,
                                kObs ? a.kin + 20 * g : nullptr, a_pre, delayed, obs_step);
    } else {
        for (int s = 0; s < a.n_sub; ++s, ++ph) {
            float4* buf = s_pos + (s & 1) * B;
            if (tile_dw) {
                buf[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
                if (warp_local) __syncwarp();
                else __syncthreads();
            }
            if (active) substep<kFlags, kN>(d, m, env.flags, buf + env.ls, env.N, t - env.ls, a.c);
        }
    }
    bool bad = false;
    if (active) {
        store_state(a.state, a.n, g, d, loops);
        a.state[5 * a.n + g] = make_float4(rpm[0], rpm[1], rpm[2], rpm[3]);
        bad = !finite_state(d);
    }
    const unsigned bad_mask = __ballot_sync(0xffffffffu, bad);
    if (bad_mask && (t & 31) == 0) {
        atomicOr(a.status, MDG_STATUS_NONFINITE);
        atomicMin(a.status + 1, (unsigned)(g + __ffs(bad_mask) - 1));
    }
    if (kObs) {
        float4* pb = s_pos + (ph & 1) * B;  // not the buffer the last substep read
        pb[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
        s_vel[t] = make_float4(d.v[0], d.v[1], d.v[2], 0.f);
        // every warp reads only its own environments' entries when the tile is warp-local
        if (warp_local) __syncwarp();
        else __syncthreads();
        // observations through per-warp staging (coalesced stores: 0.4-0.6 us less per step on
        // the 65536-drone swarm than strided ones); the randomization variant writes its noisy
        // rows directly
        if (kFlags != kFlagsDR || a.obs_host) {
            float4* stage = reinterpret_cast<float4*>(reinterpret_cast<char*>(smem) + obs_stage_offset(B)) +
                            (t >> 5) * 192;
            write_obs_staged<kN>(a, stage, active, g, t & 31, tile.first_drone + env.ls, t - env.ls, d, rpm,
                                 pb + env.ls, s_vel + env.ls, env.N);
        } else if (active) {
            if constexpr (kFlags == kFlagsDR) {  // sensor noise; delayed ones were written at the start
                if (!delayed)
                    noisy_kin(a.kin + 20 * g, d, rpm, a.rand->dr + (long long)env.id * MDG_DR_PARAMS, a.rand->seed,
                              obs_step, g, a.rand->obs_bias);
            }
            write_knn<kN>(a.nbr_idx, a.nbr_rel, g, tile.first_drone + env.ls, t - env.ls, d, pb + env.ls,
                          s_vel + env.ls, env.N);
        }
    }
}

// Shared memory of the rollout kernel (B = blockDim.x): float4 pos[2][B], float4 vel[B],
// int off[B + 1], info[B], goff[B], item.
__host__ __device__ constexpr size_t rollout_smem_bytes(int B) { return (size_t)B * 48 + (size_t)(3 * B + 2) * 4; }

// K control steps in one launch. Persistent CTAs take work items (whole environments)
// from an atomic counter; an item keeps its drones in registers for all K steps, so the
// state crosses HBM once per rollout instead of once per step. Per step: action (the
// next one prefetched), RPMs or PID, n_sub substeps, optional observations.
template <int kFlags, int kN>
__global__ void __launch_bounds__(StepBounds<kN>::threads, StepBounds<kN>::min_blocks)
    rollout_kernel(const RolloutArgs r)
{
    extern __shared__ float4 smem[];
    const StepArgs& a = r.s;
    const int B = blockDim.x;
    float4* s_pos = smem;          // [2][B]
    float4* s_vel = smem + 2 * B;  // [B]
    int* s_off = reinterpret_cast<int*>(smem + 3 * B);  // [B + 1]
    int* s_info = s_off + B + 1;                         // [B]
    int* s_goff = s_info + B;                            // [B]
    int* s_item = s_goff + B;
    const int t = threadIdx.x;
    const bool uniform = a.uniform_N > 0;
    // static schedule: this block's own list of items; else the next item from the counter
    const int sched_lo = r.sched_off ? r.sched_off[blockIdx.x] : 0;
    const int sched_hi = r.sched_off ? r.sched_off[blockIdx.x + 1] : 0;

    for (int taken = 0;; ++taken) {
        if (t == 0) {
            if (r.sched_off) {
                const int i = sched_lo + taken;
                *s_item = i < sched_hi && MDG_CHECK(i >= 0 && i < r.n_items, a.status) ? r.sched_items[i] : r.n_items;
            } else {
                *s_item = atomicAdd(r.work_counter, 1);
            }
        }
        __syncthreads();
        const int item_idx = *s_item;
        if (item_idx >= r.n_items) break;
        const int item = r.sched_off ? item_idx : r.item_order[item_idx];

        // ---- this thread's drone and environment
        int n_drones, bits;
        EnvSlot env = {0, 0, 0, 0, 0};
        long long g = 0, env_first = 0;
        if (uniform) {
            const int first_env = item * a.envs_per_tile;
            int n_envs = min(a.envs_per_tile, a.n_envs - first_env);
            if (!MDG_CHECK(item >= 0 && first_env >= 0 && n_envs >= 0 && n_envs * a.uniform_N <= B &&
                               (long long)(first_env + n_envs) * a.uniform_N <= a.n,
                           a.status))
                n_envs = 0;
            n_drones = n_envs * a.uniform_N;
            bits = a.uniform_bits;
            if (t < n_drones) {
                const int k = t / (kN > 0 ? kN : a.uniform_N);
                env.id = first_env + k;
                env.ls = k * a.uniform_N;
                env.N = a.uniform_N;
                env.flags = a.env_flags[first_env + k];
                env.act = a.act_type == MDG_ACT_MIXED ? (int)a.env_act[first_env + k] : a.act_type;
                env_first = (long long)(first_env + k) * a.uniform_N;
                g = env_first + (t - env.ls);
            }
        } else {
            const int4 it = r.items[item];
            int n_envs = it.y;
            n_drones = it.z;
            bits = it.w;
            if (!MDG_CHECK(item >= 0 && it.x >= 0 && n_envs >= 0 && n_envs <= B && n_drones >= 0 && n_drones <= B &&
                               it.x + n_envs <= a.n_envs,
                           a.status)) {
                n_envs = 0;
                n_drones = 0;
            }
            for (int i = t; i < n_envs; i += B) {
                const int e = r.slot_env[it.x + i];
                const int act = a.act_type == MDG_ACT_MIXED ? (int)a.env_act[e] : a.act_type;
                s_off[i] = r.slot_loff[it.x + i];
                s_goff[i] = r.slot_goff[it.x + i];
                s_info[i] = (int)a.env_flags[e] | (act << 8);
            }
            if (t == 0) s_off[n_envs] = n_drones;
            __syncthreads();
            if (t < n_drones) {
                int lo = 0, hi = n_envs - 1;  // largest slot with s_off[slot] <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                env.ls = s_off[lo];
                env.N = s_off[lo + 1] - env.ls;
                env.flags = s_info[lo] & 0xff;
                env.act = s_info[lo] >> 8;
                if (kFlags == kFlagsDR) env.id = r.slot_env[it.x + lo];
                env_first = s_goff[lo];
                g = env_first + (t - env.ls);
                // debug builds: the environment's drones lie inside the batch
                if (!MDG_CHECK(env_first >= 0 && env_first + env.N <= a.n, a.status)) {
                    env_first = 0;
                    g = 0;
                    env.N = 0;
                }
            }
            check_env(env, t, n_drones, a.status);
        }
        const bool active = t < n_drones && env.N > 0;  // env.N == 0 only after a failed debug check
        const bool is_pid = env.act == MDG_ACT_PID;
        const bool loops = is_pid || (runtime_variant(kFlags) && uses_loops(env.act));
        const bool tile_dw = (bits & kTileAnyDW) != 0;
        const bool warp_local = (bits & kTileWarpLocal) != 0;

        Drone d;
        {
            float4 s0 = {}, s1 = {}, s2 = {}, s3 = {}, s4 = {};
            if (active) {
                s0 = a.state[g];
                s1 = a.state[a.n + g];
                s2 = a.state[2 * a.n + g];
                s3 = a.state[3 * a.n + g];
                if (a.act_type != MDG_ACT_RPM) s4 = a.state[4 * a.n + g];
            }
            unpack_state(s0, s1, s2, s3, s4, d);
        }
        float4 act = {};
        if (active) act = a.action[g];
        float rpm[4] = {0.f, 0.f, 0.f, 0.f};
        if constexpr (kFlags == kFlagsDR) {  // the RPMs before the rollout (delayed observations)
            if (active) {
                const float4 p5 = a.state[5 * a.n + g];
                rpm[0] = p5.x, rpm[1] = p5.y, rpm[2] = p5.z, rpm[3] = p5.w;
            }
        }
        int sub = 0;  // substeps taken in this item: the snapshot buffers alternate across steps
        // roll, pitch, yaw of the current state when the previous step's observation computed
        // them (the PID of the next step reads the same state)
        float rpy_c[3] = {0.f, 0.f, 0.f};
        bool have_rpy = false;
        for (int k = 0; k < r.K; ++k) {
            const float a_pre[4] = {rpm[0], rpm[1], rpm[2], rpm[3]};  // the RPMs of the step's start
            float4 next = {};
            if (active && k + 1 < r.K) next = a.action[(k + 1) * r.action_stride + g];
            if (active) {
                if constexpr (kFlags == kFlagsDR)  // action latency
                    act = delayed_action(a, g, act, (int)a.rand->dr[(long long)env.id * MDG_DR_PARAMS + MDG_DR_DELAY]);
                if (runtime_variant(kFlags) && env.act >= MDG_ACT_RPM_NORM) {
                    ext_action_rpm(d, act, env.act, a.c, rpm);
                } else if (is_pid) {
                    float ep[3], ye;
                    const float4 wp = (runtime_variant(kFlags) && a.c.dsl) ? dsl_setpoint(d, act, a.setpoints + g, a.c) : act;
                    pid(d, wp, a.c, rpm, ep, ye, float4{}, have_rpy ? rpy_c : nullptr);
                } else {
                    rpm[0] = fminf(a.c.max_rpm, fmaxf(0.f, act.x));
                    rpm[1] = fminf(a.c.max_rpm, fmaxf(0.f, act.y));
                    rpm[2] = fminf(a.c.max_rpm, fmaxf(0.f, act.z));
                    rpm[3] = fminf(a.c.max_rpm, fmaxf(0.f, act.w));
                }
            }
            have_rpy = false;
            const Motor m = motor(rpm, a.c);
            const bool obs_now = r.obs_mode == 2 || (r.obs_mode == 1 && k == r.K - 1);
            bool delayed = false;
            unsigned long long obs_step = 0;
            if constexpr (rk4_variant(kFlags)) {
                rk4_substeps<kFlags, kN>(d, m, env, s_pos, B, t, active, tile_dw, warp_local, a.n_sub, sub, a.c);
            } else if constexpr (kFlags == kFlagsDR) {
                float* kin_row = obs_now ? a.kin + 20 * ((r.obs_mode == 2 ? (long long)k * a.n : 0) + g) : nullptr;
                randomized_substeps<kN>(a, d, rpm, env, s_pos, B, t, g, active, tile_dw, warp_local, sub, kin_row,
                                        a_pre, delayed, obs_step);
            } else {
                for (int s = 0; s < a.n_sub; ++s, ++sub) {
                    float4* buf = s_pos + (sub & 1) * B;
                    if (tile_dw) {
                        buf[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
                        if (warp_local) __syncwarp();
                        else __syncthreads();
                    }
                    if (active) substep<kFlags, kN>(d, m, env.flags, buf + env.ls, env.N, t - env.ls, a.c);
                }
            }
            if (r.obs_mode == 2 || (r.obs_mode == 1 && k == r.K - 1)) {
                const long long o = r.obs_mode == 2 ? (long long)k * a.n : 0;
                float4* pb = s_pos + (sub & 1) * B;  // not the buffer the last substep read
                pb[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
                s_vel[t] = make_float4(d.v[0], d.v[1], d.v[2], 0.f);
                if (warp_local) __syncwarp();  // a warp-local tile: each warp reads its own entries
                else __syncthreads();
                // direct strided stores: staging them through shared memory as the step kernel
                // does measured 2% slower per control step here (more registers in the loop)
                if (active) {
                    if constexpr (kFlags == kFlagsDR) {  // sensor noise; delayed ones were written at the start
                        if (!delayed)
                            noisy_kin(a.kin + 20 * (o + g), d, rpm, a.rand->dr + (long long)env.id * MDG_DR_PARAMS,
                                      a.rand->seed, obs_step, g, a.rand->obs_bias);
                    } else {
                        rpy_of(d.q, rpy_c[0], rpy_c[1], rpy_c[2]);
                        have_rpy = true;
                        write_kin(a.kin, o + g, d, rpm, rpy_c);
                    }
                    write_knn<kN>(a.nbr_idx, a.nbr_rel, o + g, env_first, t - env.ls, d, pb + env.ls,
                                  s_vel + env.ls, env.N);
                }
                if (warp_local) __syncwarp();  // the next step publishes into pb again
                else __syncthreads();
            }
            act = next;
        }
        bool bad = false;
        if (active) {
            store_state(a.state, a.n, g, d, loops);
            a.state[5 * a.n + g] = make_float4(rpm[0], rpm[1], rpm[2], rpm[3]);
            bad = !finite_state(d);
        }
        const unsigned bad_mask = __ballot_sync(0xffffffffu, bad);
        const long long g_bad = __shfl_sync(0xffffffffu, g, bad_mask ? __ffs(bad_mask) - 1 : 0);
        if (bad_mask && (t & 31) == 0) {
            atomicOr(a.status, MDG_STATUS_NONFINITE);
            atomicMin(a.status + 1, (unsigned)g_bad);
        }
        __syncthreads();  // s_item and the tables are rewritten for the next item
    }
}

__global__ void __launch_bounds__(1024) obs_kernel(const StepArgs a)
{
    extern __shared__ float4 smem[];
    const int B = blockDim.x;
    float4* s_pos = smem;
    float4* s_vel = smem + 2 * B;
    int* s_off = reinterpret_cast<int*>(smem + 3 * B);
    int* s_info = s_off + B + 1;

    const TileInfo tile = get_tile(a);
    const int t = threadIdx.x;
    const bool active = t < tile.n_drones;
    const long long g = tile.first_drone + t;
    Drone d = {};
    float4 ap = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) {
        load_state(a.state, a.n, g, d, false);
        ap = a.state[5 * a.n + g];
    }
    const EnvSlot env = tile_env(a, tile, s_off, s_info);
    s_pos[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
    s_vel[t] = make_float4(d.v[0], d.v[1], d.v[2], 0.f);
    __syncthreads();
    if (active) {
        const float apv[4] = {ap.x, ap.y, ap.z, ap.w};
        write_kin(a.kin, g, d, apv);
        write_knn<0>(a.nbr_idx, a.nbr_rel, g, tile.first_drone + env.ls, t - env.ls, d, s_pos + env.ls,
                     s_vel + env.ls, env.N);
    }
}

// ---- learned surrogate: inputs, prepare / apply around the network, fallback ----

// The 41 raw inputs of drone g: [p, q, v, w, rpm, 4 neighbours' (dp, dv)].
__device__ __forceinline__ void surrogate_inputs(const Drone& d, const float rpm[4], const float f[24], float x[41])
{
    x[0] = d.p[0]; x[1] = d.p[1]; x[2] = d.p[2];
    x[3] = d.q[0]; x[4] = d.q[1]; x[5] = d.q[2]; x[6] = d.q[3];
    x[7] = d.v[0]; x[8] = d.v[1]; x[9] = d.v[2];
    x[10] = d.w[0]; x[11] = d.w[1]; x[12] = d.w[2];
    x[13] = rpm[0]; x[14] = rpm[1]; x[15] = rpm[2]; x[16] = rpm[3];
#pragma unroll
    for (int k = 0; k < 24; ++k) x[17 + k] = f[k];
}

// Raw inputs of the current state with given RPMs (training data).
__global__ void __launch_bounds__(1024) features_kernel(const SurrogateArgs sa)
{
    extern __shared__ float4 smem[];
    const StepArgs& a = sa.s;
    const int B = blockDim.x;
    float4* s_pos = smem;
    float4* s_vel = smem + 2 * B;
    int* s_off = reinterpret_cast<int*>(smem + 3 * B);
    int* s_info = s_off + B + 1;
    const TileInfo tile = get_tile(a);
    const int t = threadIdx.x;
    const bool active = t < tile.n_drones;
    const long long g = tile.first_drone + t;
    Drone d = {};
    float4 r4 = {};
    if (active) {
        load_state(a.state, a.n, g, d, false);
        r4 = sa.rpm[g];
    }
    const EnvSlot env = tile_env(a, tile, s_off, s_info);
    s_pos[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
    s_vel[t] = make_float4(d.v[0], d.v[1], d.v[2], 0.f);
    __syncthreads();
    if (active) {
        int bi[4];
        float f[24], x[41];
        knn_best4<0>(t - env.ls, d.p, s_pos + env.ls, env.N, bi);
        knn_features(bi, d, s_pos + env.ls, s_vel + env.ls, f);
        const float rpm[4] = {r4.x, r4.y, r4.z, r4.w};
        surrogate_inputs(d, rpm, f, x);
        float* o = sa.raw + 41 * g;
#pragma unroll
        for (int k = 0; k < 41; ++k) o[k] = x[k];
    }
}

// Before the network: action -> RPMs (PID state and plane 5 updated), standardised
// inputs (bf16, zero padded to 64), and the out-of-distribution test of each drone; an
// environment with any such drone is flagged once and listed for the fallback.
__global__ void __launch_bounds__(1024) surrogate_prepare_kernel(const SurrogateArgs sa)
{
    extern __shared__ float4 smem[];
    const StepArgs& a = sa.s;
    const int B = blockDim.x;
    float4* s_pos = smem;
    float4* s_vel = smem + 2 * B;
    int* s_off = reinterpret_cast<int*>(smem + 3 * B);
    int* s_info = s_off + B + 1;
    const TileInfo tile = get_tile(a);
    const int t = threadIdx.x;
    const bool active = t < tile.n_drones;
    const long long g = tile.first_drone + t;
    float4 s0 = {}, s1 = {}, s2 = {}, s3 = {}, s4 = {}, act = {};
    if (active) {
        s0 = a.state[g];
        s1 = a.state[a.n + g];
        s2 = a.state[2 * a.n + g];
        s3 = a.state[3 * a.n + g];
        if (a.act_type != MDG_ACT_RPM) s4 = a.state[4 * a.n + g];
        act = a.action[g];
    }
    const EnvSlot env = tile_env(a, tile, s_off, s_info);
    Drone d;
    unpack_state(s0, s1, s2, s3, s4, d);
    float rpm[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
        if (uses_loops(env.act) || env.act >= MDG_ACT_RPM_NORM) {
            if (env.act == MDG_ACT_PID) {
                float ep[3], ye;
                const float4 wp = a.c.dsl ? dsl_setpoint(d, act, a.setpoints + g, a.c) : act;
                pid(d, wp, a.c, rpm, ep, ye);
            } else {
                ext_action_rpm(d, act, env.act, a.c, rpm);
            }
            if (uses_loops(env.act)) {
                a.state[3 * a.n + g] = make_float4(d.w[2], d.ip[0], d.ip[1], d.ip[2]);
                a.state[4 * a.n + g] = make_float4(d.ia[0], d.ia[1], d.ia[2], 0.f);
            }
        } else {
            rpm[0] = fminf(a.c.max_rpm, fmaxf(0.f, act.x));
            rpm[1] = fminf(a.c.max_rpm, fmaxf(0.f, act.y));
            rpm[2] = fminf(a.c.max_rpm, fmaxf(0.f, act.z));
            rpm[3] = fminf(a.c.max_rpm, fmaxf(0.f, act.w));
        }
        a.state[5 * a.n + g] = make_float4(rpm[0], rpm[1], rpm[2], rpm[3]);
    }
    s_pos[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
    s_vel[t] = make_float4(d.v[0], d.v[1], d.v[2], 0.f);
    // the normalisation (mean, 1/std, lo, hi of every input), read by every drone
    __shared__ float s_nrm[4][MDG_MLP_IN];
    for (int i = t; i < 4 * MDG_MLP_IN; i += B) {
        const int r = i / MDG_MLP_IN, k = i % MDG_MLP_IN;
        const float* src = r == 0 ? sa.in_mean : r == 1 ? sa.in_inv_std : r == 2 ? sa.in_lo : sa.in_hi;
        s_nrm[r][k] = src[k];
    }
    __syncthreads();
    bool ood = false;
    if (active) {
        int bi[4];
        float f[24], x[41];
        knn_best4<0>(t - env.ls, d.p, s_pos + env.ls, env.N, bi);
        knn_features(bi, d, s_pos + env.ls, s_vel + env.ls, f);
        surrogate_inputs(d, rpm, f, x);
        // the 128-byte input row in eight 16-byte stores of eight standardised inputs each
        uint4* row = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(sa.x) + 64 * g);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 8 * q + 2 * i;
                float z0 = 0.f, z1 = 0.f;
                if (k < 41) {
                    z0 = (x[k] - s_nrm[0][k]) * s_nrm[1][k];
                    ood = ood || !(fabsf(z0) <= sa.ood_z) || !(x[k] >= s_nrm[2][k] && x[k] <= s_nrm[3][k]);
                }
                if (k + 1 < 41) {
                    z1 = (x[k + 1] - s_nrm[0][k + 1]) * s_nrm[1][k + 1];
                    ood = ood || !(fabsf(z1) <= sa.ood_z) || !(x[k + 1] >= s_nrm[2][k + 1] && x[k + 1] <= s_nrm[3][k + 1]);
                }
                const __nv_bfloat162 zz = __floats2bfloat162_rn(z0, z1);
                o[i] = *reinterpret_cast<const uint32_t*>(&zz);
            }
            row[q] = make_uint4(o[0], o[1], o[2], o[3]);
        }
        if (ood) {
            const int e = (int)((tile.first_drone + env.ls) / env.N);  // uniform batches
            if (atomicOr(&sa.env_flag[e], 1u) == 0u) sa.fallback_list[atomicAdd(sa.fallback_count, 1)] = e;
        }
    }
}

// After the network: state += de-standardised prediction (q renormalised) for every drone
// whose environment is not flagged. Uniform batches: environment of drone g is g / N.
__global__ void __launch_bounds__(256) surrogate_apply_kernel(const SurrogateArgs sa)
{
    const StepArgs& a = sa.s;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < a.n;
         g += (long long)gridDim.x * blockDim.x) {
        if (sa.env_flag[g / a.uniform_N]) continue;
        Drone d;
        load_state(a.state, a.n, g, d, false);
        const float4* y4 = reinterpret_cast<const float4*>(sa.y + 32 * g);
        float y[16];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = y4[k];
            y[4 * k] = v.x; y[4 * k + 1] = v.y; y[4 * k + 2] = v.z; y[4 * k + 3] = v.w;
        }
        float dl[13];
#pragma unroll
        for (int k = 0; k < 13; ++k) dl[k] = sa.out_mean[k] + sa.out_std[k] * y[k];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            d.p[r] += dl[r];
            d.v[r] += dl[7 + r];
            d.w[r] += dl[10 + r];
        }
        float qn = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            d.q[r] += dl[3 + r];
            qn += d.q[r] * d.q[r];
        }
        const float inv = rsqrtf(qn);
#pragma unroll
        for (int r = 0; r < 4; ++r) d.q[r] *= inv;
        store_state(a.state, a.n, g, d, false);
    }
}

// The plain integrator for the flagged environments: one warp per environment (N <= 32),
// the RPMs the prepare step stored in plane 5, n_sub substeps with the warp's own
// position snapshot.
__global__ void __launch_bounds__(128) surrogate_fallback_kernel(const SurrogateArgs sa)
{
    __shared__ float4 s_pos[4][2][32];
    const StepArgs& a = sa.s;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int count = *sa.fallback_count;
    for (int item = blockIdx.x * 4 + wib; item < count; item += gridDim.x * 4) {
        const int e = sa.fallback_list[item];
        if (!MDG_CHECK(e >= 0 && e < a.n_envs, a.status)) continue;
        const int N = a.uniform_N;
        const bool active = lane < N;
        const long long g = (long long)e * N + lane;
        Drone d = {};
        float rpm[4] = {0.f, 0.f, 0.f, 0.f};
        if (active) {
            load_state(a.state, a.n, g, d, false);
            const float4 r = a.state[5 * a.n + g];
            rpm[0] = r.x; rpm[1] = r.y; rpm[2] = r.z; rpm[3] = r.w;
        }
        const int flags = a.env_flags[e];
        const Motor m = motor(rpm, a.c);
        for (int s = 0; s < a.n_sub; ++s) {
            float4* buf = s_pos[wib][s & 1];
            buf[lane] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
            __syncwarp();
            if (active) substep<kFlagsGndRotor, -1>(d, m, flags, buf, N, lane, a.c);
        }
        if (active) {
            store_state(a.state, a.n, g, d, false);
            if (!finite_state(d)) {
                atomicOr(a.status, MDG_STATUS_NONFINITE);
                atomicMin(a.status + 1, (unsigned)g);
            }
        }
        __syncwarp();
    }
}

// The plain integrator for the flagged environments of larger size or with Runge-Kutta
// substeps: one block per listed environment (blockDim = N rounded up to 32), the RPMs the
// prepare step stored in plane 5, n_sub substeps with the block's position snapshot.
template <bool kRK4>
__global__ void __launch_bounds__(1024) surrogate_fallback_block_kernel(const SurrogateArgs sa)
{
    extern __shared__ float4 smem[];
    float4* s_pos = smem;  // [2][B]
    const StepArgs& a = sa.s;
    const int t = threadIdx.x, B = blockDim.x;
    const int count = *sa.fallback_count;
    for (int item = blockIdx.x; item < count; item += gridDim.x) {
        const int e = sa.fallback_list[item];
        if (!MDG_CHECK(e >= 0 && e < a.n_envs && a.uniform_N <= B, a.status)) continue;
        const int N = a.uniform_N;
        const bool active = t < N;
        const long long g = (long long)e * N + t;
        Drone d = {};
        float rpm[4] = {0.f, 0.f, 0.f, 0.f};
        if (active) {
            load_state(a.state, a.n, g, d, false);
            const float4 r = a.state[5 * a.n + g];
            rpm[0] = r.x; rpm[1] = r.y; rpm[2] = r.z; rpm[3] = r.w;
        }
        EnvSlot env = {0, N, (int)a.env_flags[e], 0, e};
        const Motor m = motor(rpm, a.c);
        const bool dw = (env.flags & MDG_DW) != 0;
        int ph = 0;
        if constexpr (kRK4) {
            rk4_substeps<kFlagsRK4, -1>(d, m, env, s_pos, B, t, active, dw, false, a.n_sub, ph, a.c);
        } else {
            for (int s = 0; s < a.n_sub; ++s, ++ph) {
                float4* buf = s_pos + (ph & 1) * B;
                if (dw) {
                    buf[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
                    __syncthreads();
                }
                if (active) substep<kFlagsGndRotor, -1>(d, m, env.flags, buf, N, t, a.c);
            }
        }
        if (active) {
            store_state(a.state, a.n, g, d, false);
            if (!finite_state(d)) {
                atomicOr(a.status, MDG_STATUS_NONFINITE);
                atomicMin(a.status + 1, (unsigned)g);
            }
        }
        __syncthreads();  // the snapshot is rewritten for the next environment
    }
}

__global__ void __launch_bounds__(256) pid_kernel(const PidArgs a)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < a.n;
         g += (long long)gridDim.x * blockDim.x) {
        Drone d;
        load_state(a.state, a.n, g, d, true);
        float rpm[4], ep[3], ye;
        float4 wp = a.waypoints[g];
        if (a.c.dsl) wp = dsl_setpoint(d, wp, a.setpoints + g, a.c);
        if (a.target_acc) pid<true>(d, wp, a.c, rpm, ep, ye, a.target_acc[g]);
        else pid(d, wp, a.c, rpm, ep, ye);
        a.rpm_out[g] = make_float4(rpm[0], rpm[1], rpm[2], rpm[3]);
        a.state[3 * a.n + g] = make_float4(d.w[2], d.ip[0], d.ip[1], d.ip[2]);
        a.state[4 * a.n + g] = make_float4(d.ia[0], d.ia[1], d.ia[2], 0.f);
        if (a.pos_err) {
            a.pos_err[3 * g + 0] = ep[0];
            a.pos_err[3 * g + 1] = ep[1];
            a.pos_err[3 * g + 2] = ep[2];
        }
        if (a.yaw_err) a.yaw_err[g] = ye;
    }
}

}  // namespace

// The step-kernel variants: compile-time physics subset and environment size for the
// uniform batches of the benchmark workloads, and a runtime-generic one for the rest.
// (physics flags, environment size): kFlags 0-7 a compile-time physics subset, 8 the
// runtime flags, kFlagsRK4 the runtime flags with Runge-Kutta substeps, kFlagsGndRotor
// the runtime flags with per-rotor ground heights, kFlagsDR the runtime flags under
// randomization, kFlagsRK4Fixed + s Runge-Kutta with the compile-time subset s; kN > 0 a
// compile-time environment size, -1 a runtime size in blocks of at most kSmallBlock
// threads, 0 any block size. The first variant that fits a launch is taken.
#define MDG_STEP_VARIANTS(X) \
    X(7, 4) X(7, 64) X(3, 1) X(8, -1) X(8, 0) X(9, -1) X(9, 0) X(10, -1) X(10, 0) X(11, 4) X(11, -1) X(11, 0) X(23, 4)

template <bool kObs>
static void* step_kernel_ptr(int flags, int N, int block)
{
#define MDG_PICK(F, NN)                                                                       \
    if ((flags == F || (F == 8 && flags < 8)) &&                                                                    \
        (NN == 0 || (block <= kSmallBlock && (NN == -1 || N == NN))))                         \
        return (void*)step_kernel<kObs, F, NN>;
    MDG_STEP_VARIANTS(MDG_PICK)
#undef MDG_PICK
    return nullptr;
}

// Opt the tile kernels in to the shared memory of the largest block, once per device.
static cudaError_t tile_kernels_setup()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    const int smem = (int)(obs_stage_offset(1024) + obs_stage_bytes(1024));
#define MDG_ATTR(F, NN)                                                                                     \
    if ((e = cudaFuncSetAttribute(step_kernel<true, F, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                  smem)) != cudaSuccess ||                                                  \
        (e = cudaFuncSetAttribute(step_kernel<false, F, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                  smem)) != cudaSuccess)                                                    \
        return e;
    MDG_STEP_VARIANTS(MDG_ATTR)
#undef MDG_ATTR
    if ((e = cudaFuncSetAttribute(obs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
    return cudaSuccess;
}

// The kernel variant (flags, N) of a launch: randomization, Runge-Kutta substeps (a
// compile-time all-effects variant for uniform batches without runtime-only features, else
// the runtime one) and per-rotor ground heights first; uniform_flags is the batch's physics
// subset, or 8 when a runtime-only feature (action types, the DSL controller) is in use.
static void variant_of(const StepArgs& a, int uniform_flags, int& flags, int& N)
{
    N = a.uniform_N;
    if (a.rand) {
        flags = kFlagsDR;
    } else if (a.c.rk4) {
        const bool fixed = uniform_flags >= 0 && uniform_flags < 8 && !a.c.gnd_rotor;
        flags = fixed ? kFlagsRK4Fixed + uniform_flags : kFlagsRK4;
        if (!fixed) N = -1;
    } else {
        flags = a.c.gnd_rotor ? kFlagsGndRotor : uniform_flags;
    }
}

cudaError_t launch_step(const StepArgs& a, int n_tiles, int block, bool with_obs, int uniform_flags, cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    cudaError_t e = tile_kernels_setup();
    if (e != cudaSuccess) return e;
    // a compile-time variant needs one physics subset and one environment size for the
    // batch; randomization, Runge-Kutta substeps (without a compile-time variant for the
    // batch) and per-rotor ground heights run in runtime-flag variants of their own
    int flags, N;
    variant_of(a, uniform_flags, flags, N);
    void* fn = with_obs ? step_kernel_ptr<true>(flags, N, block) : step_kernel_ptr<false>(flags, N, block);
    if (!fn && flags >= kFlagsRK4Fixed) {  // no compile-time Runge-Kutta variant for this size or block
        flags = kFlagsRK4;
        N = -1;
        fn = with_obs ? step_kernel_ptr<true>(flags, N, block) : step_kernel_ptr<false>(flags, N, block);
    }
    void* args[] = {const_cast<StepArgs*>(&a)};
    const size_t smem = with_obs && (flags != kFlagsDR || a.obs_host) ? obs_stage_offset(block) + obs_stage_bytes(block)
                                                                      : tile_smem_bytes(block);
    return cudaLaunchKernel(fn, dim3(n_tiles), dim3(block), args, smem, s);
}


static void* rollout_kernel_ptr(int flags, int N, int block)
{
#define MDG_PICK(F, NN)                                                                       \
    if ((flags == F || (F == 8 && flags < 8)) &&                                                                    \
        (NN == 0 || (block <= kSmallBlock && (NN == -1 || N == NN))))                         \
        return (void*)rollout_kernel<F, NN>;
    MDG_STEP_VARIANTS(MDG_PICK)
#undef MDG_PICK
    return nullptr;
}

static cudaError_t rollout_setup()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    const int smem = (int)rollout_smem_bytes(1024);
#define MDG_ATTR(F, NN)                                                                                    \
    if ((e = cudaFuncSetAttribute(rollout_kernel<F, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                  smem)) != cudaSuccess)                                                   \
        return e;
    MDG_STEP_VARIANTS(MDG_ATTR)
#undef MDG_ATTR
    if (dev >= 0 && dev < 64) done[dev] = true;
    return cudaSuccess;
}

// The rollout kernel of a launch (the step kernel's variant choice, with the same fallback).
static void* rollout_kernel_for(const StepArgs& a, int uniform_flags, int block)
{
    int flags, N;
    variant_of(a, uniform_flags, flags, N);
    void* fn = rollout_kernel_ptr(flags, N, block);
    if (!fn && flags >= kFlagsRK4Fixed) fn = rollout_kernel_ptr(kFlagsRK4, -1, block);
    return fn;
}

int rollout_blocks_per_sm(const StepArgs& a, int block, int uniform_flags)
{
    if (rollout_setup() != cudaSuccess) return 1;
    int n = 0;
    void* fn = rollout_kernel_for(a, uniform_flags, block);
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, rollout_smem_bytes(block)) != cudaSuccess ||
        n < 1)
        return 1;
    return n;
}
cudaError_t launch_rollout(const RolloutArgs& r, int block, int uniform_flags, int grid, cudaStream_t s)
{
    if (r.n_items == 0 || r.K == 0) return cudaSuccess;
    cudaError_t e = rollout_setup();
    if (e != cudaSuccess) return e;
    void* fn = rollout_kernel_for(r.s, uniform_flags, block);
    if (!fn) return cudaErrorInvalidConfiguration;
    if (grid <= 0 || grid > r.n_items) grid = r.n_items;
    void* args[] = {const_cast<RolloutArgs*>(&r)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, rollout_smem_bytes(block), s);
}

cudaError_t launch_features(const SurrogateArgs& a, int n_tiles, int block, cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    const size_t smem = tile_smem_bytes(block);
    cudaError_t e = cudaFuncSetAttribute(features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    features_kernel<<<n_tiles, block, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_prepare(const SurrogateArgs& a, int n_tiles, int block, cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    const size_t smem = tile_smem_bytes(block);
    cudaError_t e =
        cudaFuncSetAttribute(surrogate_prepare_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    surrogate_prepare_kernel<<<n_tiles, block, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reset(const ResetArgs& r, cudaStream_t s)
{
    if (r.n == 0) return cudaSuccess;
    reset_kernel<<<(unsigned)((r.n + 255) / 256), 256, 0, s>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_apply(const SurrogateArgs& a, cudaStream_t s)
{
    if (a.s.n == 0) return cudaSuccess;
    long long blocks = (a.s.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    surrogate_apply_kernel<<<(int)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_fallback(const SurrogateArgs& a, cudaStream_t s)
{
    if (a.s.n == 0) return cudaSuccess;
    const int N = a.s.uniform_N;
    if (N <= 32 && !a.s.c.rk4) {  // one warp per environment
        int blocks = (a.s.n_envs + 3) / 4;
        if (blocks > 152 * 8) blocks = 152 * 8;
        surrogate_fallback_kernel<<<blocks, 128, 0, s>>>(a);
        return cudaGetLastError();
    }
    // one block per environment, grid-stride over the listed environments
    const int B = (N + 31) / 32 * 32;
    int blocks = a.s.n_envs < 152 * 4 ? a.s.n_envs : 152 * 4;
    const size_t smem = (size_t)2 * B * sizeof(float4);
    if (a.s.c.rk4) surrogate_fallback_block_kernel<true><<<blocks, B, smem, s>>>(a);
    else surrogate_fallback_block_kernel<false><<<blocks, B, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_obs(const StepArgs& a, int n_tiles, int block, cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    cudaError_t e = tile_kernels_setup();
    if (e != cudaSuccess) return e;
    obs_kernel<<<n_tiles, block, tile_smem_bytes(block), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pid(const PidArgs& a, cudaStream_t s)
{
    if (a.n == 0) return cudaSuccess;
    long long blocks = (a.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    pid_kernel<<<(int)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mdg
