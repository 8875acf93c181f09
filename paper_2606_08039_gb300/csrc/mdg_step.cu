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

__device__ __forceinline__ void store_state(float4* __restrict__ S, long long n, long long g, const Drone& d,
                                            bool att_int)
{
    S[g] = make_float4(d.p[0], d.p[1], d.p[2], d.q[0]);
    S[n + g] = make_float4(d.q[1], d.q[2], d.q[3], d.v[0]);
    S[2 * n + g] = make_float4(d.v[1], d.v[2], d.w[0], d.w[1]);
    S[3 * n + g] = make_float4(d.w[2], d.ip[0], d.ip[1], d.ip[2]);
    if (att_int) S[4 * n + g] = make_float4(d.ia[0], d.ia[1], d.ia[2], 0.f);
}

// Body-to-world rotation matrix of a unit quaternion [w, x, y, z] (row-major).
__device__ __forceinline__ void rotation(const float q[4], float R[9])
{
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    const float xx = x * x, yy = y * y, zz = z * z;
    const float xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
    R[0] = 1.f - 2.f * (yy + zz); R[1] = 2.f * (xy - wz);        R[2] = 2.f * (xz + wy);
    R[3] = 2.f * (xy + wz);        R[4] = 1.f - 2.f * (xx + zz); R[5] = 2.f * (yz - wx);
    R[6] = 2.f * (xz - wy);        R[7] = 2.f * (yz + wx);        R[8] = 1.f - 2.f * (xx + yy);
}

// Roll, pitch, yaw in the ZYX convention.
__device__ __forceinline__ void rpy_of(const float q[4], float& roll, float& pitch, float& yaw)
{
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    roll = atan2f(2.f * (w * x + y * z), 1.f - 2.f * (x * x + y * y));
    pitch = asinf(fminf(1.f, fmaxf(-1.f, 2.f * (w * y - z * x))));
    yaw = atan2f(2.f * (w * z + x * y), 1.f - 2.f * (y * y + z * z));
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
    m.tau[0] = c.l_sqrt2 * ((f0 + f1) - (f2 + f3));
    m.tau[1] = c.l_sqrt2 * ((f1 + f2) - (f0 + f3));
    m.tau[2] = c.km * ((n1 + n3) - (n0 + n2));
    m.wsum = c.drag_k * ((n[0] + n[1]) + (n[2] + n[3]));
    return m;
}

// Cascaded PID of Section 4.2.1 (position PID -> T = m |a*| and small-angle attitude
// target -> attitude PID -> inverse mixing). The mixing rows [1,1,1,1], [1,1,-1,-1],
// [-1,1,1,-1], [-1,1,-1,1] are mutually orthogonal with squared norm 4, so the solve of
// M f = [T, tau] is f = 1/4 (T + sqrt2/L tau_x r1 + sqrt2/L tau_y r2 + k_f/k_m tau_z r3).
__device__ __forceinline__ void pid(Drone& d, const float4 wp, const DevConsts& c, float rpm[4], float ep[3],
                                    float& yaw_err)
{
    const float tgt[3] = {wp.x, wp.y, wp.z};
    float acc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        ep[r] = tgt[r] - d.p[r];
        d.ip[r] = fminf(c.pos_iclamp, fmaxf(-c.pos_iclamp, d.ip[r] + ep[r] * c.dt_ctrl));
        acc[r] = c.pos_kp[r] * ep[r] + c.pos_ki[r] * d.ip[r] - c.pos_kd[r] * d.v[r];
    }
    acc[2] += c.g;
    const float T = c.mass * sqrtf(acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2]);
    float sps, cps;
    sincosf(wp.w, &sps, &cps);
    const float phi_t = (acc[0] * sps - acc[1] * cps) / c.g;
    const float theta_t = (acc[0] * cps + acc[1] * sps) / c.g;
    float roll, pitch, yaw;
    rpy_of(d.q, roll, pitch, yaw);
    float e[3] = {phi_t - roll, theta_t - pitch, wp.w - yaw};
    e[2] -= 2.f * kPi * floorf((e[2] + kPi) * (0.5f / kPi));  // wrap to [-pi, pi)
    float tau[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        d.ia[r] = fminf(c.att_iclamp, fmaxf(-c.att_iclamp, d.ia[r] + e[r] * c.dt_ctrl));
        tau[r] = c.att_kp[r] * e[r] + c.att_ki[r] * d.ia[r] - c.att_kd[r] * d.w[r];
    }
    const float tx = tau[0] * c.alloc_xy, ty = tau[1] * c.alloc_xy, tz = tau[2] * c.alloc_z;
    const float f[4] = {0.25f * (T + tx - ty - tz), 0.25f * (T + tx + ty + tz), 0.25f * (T - tx + ty - tz),
                        0.25f * (T - tx - ty + tz)};
#pragma unroll
    for (int i = 0; i < 4; ++i) rpm[i] = sqrtf(fminf(c.f_max, fmaxf(0.f, f[i])) * c.inv_kf);
    yaw_err = e[2];
}

// One substep: forces of Eq. motor/ground/drag/downwash, Newton-Euler, forward Euler
// and the exponential map (all from the start-of-substep state). `env_pos` points at
// the shared-memory positions of this drone's environment (N entries).
__device__ __forceinline__ void substep(Drone& d, const Motor& m, int flags, const float4* env_pos, int N,
                                        const DevConsts& c)
{
    float R[9];
    rotation(d.q, R);
    float F[3] = {R[2] * m.T, R[5] * m.T, R[8] * m.T - c.mass * c.g};
    if (flags & MDG_GND) {
        // gate |roll| < pi/2 and |pitch| < pi/2: cos(roll) cos(pitch) = R22 > 0, |sin(pitch)| = |R20| < 1
        if (R[8] > 0.f && fabsf(R[6]) < 1.f) {
            const float h = fmaxf(d.p[2], c.h_clip);
            F[2] += c.gnd_k * m.T / (h * h);
        }
    }
    if (flags & MDG_DRAG) {
        const float vb0 = R[0] * d.v[0] + R[3] * d.v[1] + R[6] * d.v[2];
        const float vb1 = R[1] * d.v[0] + R[4] * d.v[1] + R[7] * d.v[2];
        const float vb2 = R[2] * d.v[0] + R[5] * d.v[1] + R[8] * d.v[2];
        const float fb0 = -m.wsum * c.c_xy * vb0, fb1 = -m.wsum * c.c_xy * vb1, fb2 = -m.wsum * c.c_z * vb2;
        F[0] += R[0] * fb0 + R[1] * fb1 + R[2] * fb2;
        F[1] += R[3] * fb0 + R[4] * fb1 + R[5] * fb2;
        F[2] += R[6] * fb0 + R[7] * fb1 + R[8] * fb2;
    }
    if (flags & MDG_DW) {
        // Sum over drones strictly above (dz > dz_min >= 0, which also skips this drone)
        // within the lateral cut-off of C1 (r_p/(4 dz))^2 exp(-dxy^2 / (2 beta^2)),
        // beta = C2 dz + C3. One reciprocal r = 1/(dz^2 beta^2) gives both 1/dz^2 = beta^2 r
        // and 1/beta^2 = dz^2 r; beta^2 is floored at 1e-12.
        const float px = d.p[0], py = d.p[1], pz = d.p[2];
        float acc = 0.f;
        for (int k = 0; k < N; ++k) {
            const float4 o = env_pos[k];
            const float dz = o.z - pz;
            if (dz > c.dw_dz_min) {
                const float dx = o.x - px, dy = o.y - py;
                const float d2 = dx * dx + dy * dy;
                if (d2 < c.dw_max_xy2) {
                    const float beta = fmaf(c.dw_c2, dz, c.dw_c3);
                    const float b2 = fmaxf(beta * beta, 1e-12f);
                    const float dz2 = dz * dz;
                    const float r = rcp_approx(dz2 * b2);
                    const float e = ex2_approx(-0.72134752044448170368f * d2 * dz2 * r);  // -0.5 log2(e)
                    acc += (e > 0.f) ? c.dw_k * b2 * r * e : 0.f;
                }
            }
        }
        F[2] -= acc;
    }
    // Newton-Euler: omega_dot = J^-1 (tau - omega x (J omega)), omega in the body frame
    const float Jw0 = c.J[0] * d.w[0], Jw1 = c.J[1] * d.w[1], Jw2 = c.J[2] * d.w[2];
    const float wd0 = c.inv_J[0] * (m.tau[0] - (d.w[1] * Jw2 - d.w[2] * Jw1));
    const float wd1 = c.inv_J[1] * (m.tau[1] - (d.w[2] * Jw0 - d.w[0] * Jw2));
    const float wd2 = c.inv_J[2] * (m.tau[2] - (d.w[0] * Jw1 - d.w[1] * Jw0));
    const float dt = c.dt_sim;
    // exponential map with the old body rate: q <- q (x) [cos(|w| dt/2), sin(|w| dt/2) w/|w|]
    const float nw2 = d.w[0] * d.w[0] + d.w[1] * d.w[1] + d.w[2] * d.w[2];
    if (nw2 > 0.f) {
        const float nw = sqrtf(nw2);
        float s, co;
        sincosf(0.5f * dt * nw, &s, &co);
        const float k = s / nw;
        const float bx = k * d.w[0], by = k * d.w[1], bz = k * d.w[2];
        const float w = d.q[0], x = d.q[1], y = d.q[2], z = d.q[3];
        float qw = w * co - x * bx - y * by - z * bz;
        float qx = w * bx + x * co + y * bz - z * by;
        float qy = w * by - x * bz + y * co + z * bx;
        float qz = w * bz + x * by - y * bx + z * co;
        const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        d.q[0] = qw * inv; d.q[1] = qx * inv; d.q[2] = qy * inv; d.q[3] = qz * inv;
    } else {
        const float inv = rsqrtf(d.q[0] * d.q[0] + d.q[1] * d.q[1] + d.q[2] * d.q[2] + d.q[3] * d.q[3]);
#pragma unroll
        for (int r = 0; r < 4; ++r) d.q[r] *= inv;
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

__device__ __forceinline__ bool finite_state(const Drone& d)
{
    bool ok = true;
#pragma unroll
    for (int r = 0; r < 3; ++r) ok = ok && isfinite(d.p[r]) && isfinite(d.v[r]) && isfinite(d.w[r]);
#pragma unroll
    for (int r = 0; r < 4; ++r) ok = ok && isfinite(d.q[r]);
    return ok;
}

// KIN observation [p, q, roll/pitch/yaw, v, w, a_prev] as five float4 stores.
__device__ __forceinline__ void write_kin(float* __restrict__ kin, long long g, const Drone& d, const float a[4])
{
    float roll, pitch, yaw;
    rpy_of(d.q, roll, pitch, yaw);
    float4* o = reinterpret_cast<float4*>(kin + 20 * g);
    o[0] = make_float4(d.p[0], d.p[1], d.p[2], d.q[0]);
    o[1] = make_float4(d.q[1], d.q[2], d.q[3], roll);
    o[2] = make_float4(pitch, yaw, d.v[0], d.v[1]);
    o[3] = make_float4(d.v[2], d.w[0], d.w[1], d.w[2]);
    o[4] = make_float4(a[0], a[1], a[2], a[3]);
}

// The 4 nearest other drones of the environment (squared distance rounded in the
// order ((dx*dx + dy*dy) + dz*dz) without contraction, ties to the lower index),
// from the shared-memory positions/velocities of the environment.
__device__ __forceinline__ void write_knn(int4* __restrict__ nbr_idx, float* __restrict__ nbr_rel, long long g,
                                          long long env_first, int j, const Drone& d, const float4* env_pos,
                                          const float4* env_vel, int N)
{
    float bd[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
    int bi[4] = {-1, -1, -1, -1};
    for (int k = 0; k < N; ++k) {
        if (k == j) continue;
        const float4 o = env_pos[k];
        const float dx = __fsub_rn(o.x, d.p[0]), dy = __fsub_rn(o.y, d.p[1]), dz = __fsub_rn(o.z, d.p[2]);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        if (d2 < bd[3]) {
            if (d2 < bd[2]) {
                bd[3] = bd[2]; bi[3] = bi[2];
                if (d2 < bd[1]) {
                    bd[2] = bd[1]; bi[2] = bi[1];
                    if (d2 < bd[0]) {
                        bd[1] = bd[0]; bi[1] = bi[0];
                        bd[0] = d2; bi[0] = k;
                    } else {
                        bd[1] = d2; bi[1] = k;
                    }
                } else {
                    bd[2] = d2; bi[2] = k;
                }
            } else {
                bd[3] = d2; bi[3] = k;
            }
        }
    }
    int4 idx;
    idx.x = bi[0] >= 0 ? (int)(env_first + bi[0]) : -1;
    idx.y = bi[1] >= 0 ? (int)(env_first + bi[1]) : -1;
    idx.z = bi[2] >= 0 ? (int)(env_first + bi[2]) : -1;
    idx.w = bi[3] >= 0 ? (int)(env_first + bi[3]) : -1;
    nbr_idx[g] = idx;
    if (nbr_rel) {
        float4* o = reinterpret_cast<float4*>(nbr_rel + 24 * g);
        float f[24];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (bi[s] >= 0) {
                const float4 pp = env_pos[bi[s]], vv = env_vel[bi[s]];
                f[6 * s + 0] = pp.x - d.p[0]; f[6 * s + 1] = pp.y - d.p[1]; f[6 * s + 2] = pp.z - d.p[2];
                f[6 * s + 3] = vv.x - d.v[0]; f[6 * s + 4] = vv.y - d.v[1]; f[6 * s + 5] = vv.z - d.v[2];
            } else {
#pragma unroll
                for (int r = 0; r < 6; ++r) f[6 * s + r] = 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
    }
}

// Shared-memory layout of the tile kernels (B = blockDim.x):
//   float4 pos[2][B] (double-buffered substep snapshot), float4 vel[B],
//   int off[B + 1] (tile-relative env offsets), int info[B] (flags | action type << 8)
__host__ __device__ constexpr size_t tile_smem_bytes(int B) { return (size_t)B * 48 + (size_t)(2 * B + 1) * 4; }

// Loads the tile's environment table into shared memory and finds this thread's
// environment: local first drone, size, flags and action type.
struct EnvSlot {
    int ls, N, flags, act;
};

__device__ __forceinline__ EnvSlot tile_env(const StepArgs& a, const Tile& tile, int* s_off, int* s_info)
{
    const int B = blockDim.x;
    for (int i = threadIdx.x; i <= tile.w; i += B) s_off[i] = a.env_off[tile.z + i] - tile.x;
    for (int i = threadIdx.x; i < tile.w; i += B) {
        const int act = a.act_type == MDG_ACT_MIXED ? (int)a.env_act[tile.z + i] : a.act_type;
        s_info[i] = (int)a.env_flags[tile.z + i] | (act << 8);
    }
    __syncthreads();
    EnvSlot e = {0, 0, 0, 0};
    const int t = threadIdx.x;
    if (t < tile.y) {
        int lo = 0, hi = tile.w - 1;  // largest env with s_off[env] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        e.ls = s_off[lo];
        e.N = s_off[lo + 1] - e.ls;
        e.flags = s_info[lo] & 0xff;
        e.act = s_info[lo] >> 8;
    }
    return e;
}

template <bool kObs>
__global__ void __launch_bounds__(1024) step_kernel(const StepArgs a)
{
    extern __shared__ float4 smem[];
    const int B = blockDim.x;
    float4* s_pos = smem;          // [2][B]
    float4* s_vel = smem + 2 * B;  // [B]
    int* s_off = reinterpret_cast<int*>(smem + 3 * B);
    int* s_info = s_off + B + 1;

    const Tile tile = a.tiles[blockIdx.x];
    const EnvSlot env = tile_env(a, tile, s_off, s_info);
    const int t = threadIdx.x;
    const bool active = t < tile.y;
    const long long g = (long long)tile.x + t;
    const bool is_pid = env.act == MDG_ACT_PID;

    Drone d = {};
    float rpm[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
        load_state(a.state, a.n, g, d, is_pid);
        const float4 act = a.action[g];
        if (is_pid) {
            float ep[3], ye;
            pid(d, act, a.c, rpm, ep, ye);
        } else {
            rpm[0] = fminf(a.c.max_rpm, fmaxf(0.f, act.x));
            rpm[1] = fminf(a.c.max_rpm, fmaxf(0.f, act.y));
            rpm[2] = fminf(a.c.max_rpm, fmaxf(0.f, act.z));
            rpm[3] = fminf(a.c.max_rpm, fmaxf(0.f, act.w));
        }
    }
    const Motor m = motor(rpm, a.c);
    const bool tile_dw = __syncthreads_or(active && (env.flags & MDG_DW));
    for (int s = 0; s < a.n_sub; ++s) {
        float4* buf = s_pos + (s & 1) * B;
        if (tile_dw) {
            buf[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
            __syncthreads();
        }
        if (active) substep(d, m, env.flags, buf + env.ls, env.N, a.c);
    }
    bool bad = false;
    if (active) {
        store_state(a.state, a.n, g, d, is_pid);
        a.state[5 * a.n + g] = make_float4(rpm[0], rpm[1], rpm[2], rpm[3]);
        bad = !finite_state(d);
    }
    const unsigned bad_mask = __ballot_sync(0xffffffffu, bad);
    if (bad_mask && (t & 31) == 0) {
        atomicOr(a.status, MDG_STATUS_NONFINITE);
        atomicMin(a.status + 1, (unsigned)(g + __ffs(bad_mask) - 1));
    }
    if (kObs) {
        float4* pb = s_pos + (a.n_sub & 1) * B;  // not the buffer the last substep read
        pb[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
        s_vel[t] = make_float4(d.v[0], d.v[1], d.v[2], 0.f);
        __syncthreads();
        if (active) {
            write_kin(a.kin, g, d, rpm);
            write_knn(a.nbr_idx, a.nbr_rel, g, (long long)tile.x + env.ls, t - env.ls, d, pb + env.ls,
                      s_vel + env.ls, env.N);
        }
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

    const Tile tile = a.tiles[blockIdx.x];
    const EnvSlot env = tile_env(a, tile, s_off, s_info);
    const int t = threadIdx.x;
    const bool active = t < tile.y;
    const long long g = (long long)tile.x + t;
    Drone d = {};
    float4 ap = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) {
        load_state(a.state, a.n, g, d, false);
        ap = a.state[5 * a.n + g];
    }
    s_pos[t] = make_float4(d.p[0], d.p[1], d.p[2], 0.f);
    s_vel[t] = make_float4(d.v[0], d.v[1], d.v[2], 0.f);
    __syncthreads();
    if (active) {
        const float apv[4] = {ap.x, ap.y, ap.z, ap.w};
        write_kin(a.kin, g, d, apv);
        write_knn(a.nbr_idx, a.nbr_rel, g, (long long)tile.x + env.ls, t - env.ls, d, s_pos + env.ls,
                  s_vel + env.ls, env.N);
    }
}

__global__ void __launch_bounds__(256) pid_kernel(const PidArgs a)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < a.n;
         g += (long long)gridDim.x * blockDim.x) {
        Drone d;
        load_state(a.state, a.n, g, d, true);
        float rpm[4], ep[3], ye;
        pid(d, a.waypoints[g], a.c, rpm, ep, ye);
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

cudaError_t launch_step(const StepArgs& a, int n_tiles, int block, bool with_obs, cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    const size_t smem = tile_smem_bytes(block);
    if (with_obs) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        step_kernel<true><<<n_tiles, block, smem, s>>>(a);
    } else {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        step_kernel<false><<<n_tiles, block, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_obs(const StepArgs& a, int n_tiles, int block, cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    const size_t smem = tile_smem_bytes(block);
    cudaError_t e = cudaFuncSetAttribute(obs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    obs_kernel<<<n_tiles, block, smem, s>>>(a);
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
