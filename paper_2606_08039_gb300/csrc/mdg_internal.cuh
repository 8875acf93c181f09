// Internal declarations shared by the host API (mdg_api.cu) and the kernels (mdg_step.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mdg.h"

namespace mdg {

// Float32 copies of the model constants with the products the kernels need folded in
// once on the host (in double precision, then rounded).
struct DevConsts {
    float mass, inv_mass, g, inv_g;
    float kf, km, l_sqrt2;            // Eq. motor: k_f, k_m, L/sqrt(2)
    float J[3], inv_J[3];
    float gnd_k;                      // Eq. ground: C_gnd (r_p/4)^2
    float h_clip;
    float drag_k;                     // Eq. drag: 2 pi / 60 (RPM -> rad/s)
    float c_xy, c_z, c_dz;            // c_dz = c_z - c_xy
    float dw_k;                       // Eq. downwash: C1 (r_p/4)^2
    float dw_c2, dw_c3, dw_max_xy2, dw_dz_min;
    float pos_kp[3], pos_ki[3], pos_kd[3], pos_iclamp;
    float att_kp[3], att_ki[3], att_kd[3], att_iclamp;
    float dt_sim, dt_ctrl;
    float max_rpm, f_max, inv_kf;     // PID output clip: f_i in [0, k_f MAX_RPM^2]
    float alloc_xy, alloc_z;          // inverse mixing: sqrt(2)/L and k_f/k_m
};

// A launch tile: whole environments packed into one thread block.
// x = first drone, y = drones, z = first environment,
// w = environments (low 16 bits) | kTileAnyDW | kTileWarpLocal.
typedef int4 Tile;
constexpr int kTileEnvMask = 0xffff;
constexpr int kTileAnyDW = 1 << 30;      // some environment of the tile has downwash on
constexpr int kTileWarpLocal = 1 << 29;  // every environment lies inside one warp

struct StepArgs {
    float4* state;            // [6][n] float4 planes
    const float4* action;     // [n]
    float* kin;               // [n][20] or null
    int4* nbr_idx;            // [n] or null
    float* nbr_rel;           // [n][24] or null
    const Tile* tiles;
    const int32_t* env_off;   // [n_envs + 1]
    const uint8_t* env_flags; // [n_envs]
    const uint8_t* env_act;   // [n_envs] (MIXED) or null
    uint32_t* status;         // [2]: bits, first bad drone
    long long n;
    int n_sub;
    int act_type;             // MDG_ACT_RPM / PID / MIXED
    int n_envs;
    int uniform_N;            // > 0: every environment has this many drones (arithmetic tiles)
    int envs_per_tile;        // uniform batches: environments per block
    int uniform_bits;         // uniform batches: kTileAnyDW | kTileWarpLocal for every tile
    DevConsts c;
};

// A multi-step rollout (persistent kernel): K control steps per launch, tiles pulled
// from an atomic work counter. For batches of uneven environments the work items are
// built from environments sorted by (size, physics subset): slot i of the sorted order
// is environment slot_env[i], whose drones start at global index slot_goff[i] and at
// item-local index slot_loff[i].
struct RolloutArgs {
    StepArgs s;                 // action = base of [K][n] (or [n] with action_stride 0)
    long long action_stride;    // float4s between the actions of consecutive steps (n or 0)
    int K;
    int obs_mode;               // 0: none, 1: after the last step, 2: after every step ([K][n] outputs)
    int n_items;
    int* work_counter;          // zeroed before the launch
    const int* item_order;      // work items in decreasing cost
    const int4* items;          // uneven batches: {first slot, envs, drones, tile bits}
    const int* slot_env;
    const int* slot_goff;
    const int* slot_loff;
};

struct PidArgs {
    float4* state;
    const float4* waypoints;
    float4* rpm_out;
    float* pos_err;           // [n][3] or null
    float* yaw_err;           // [n] or null
    long long n;
    DevConsts c;
};

// uniform_flags: the physics subset shared by every environment, or -1 if they differ.
// Host-side builders (mdg_api.cu).
void set_last_error(const char* msg);  // the message mdg_last_error() returns on this thread
bool constants_valid(const mdg_constants& c, std::string& why);
DevConsts make_dev_consts(const mdg_constants& c);
std::vector<Tile> build_tiles(const std::vector<int32_t>& off, const std::vector<uint8_t>& flags, int block);
int default_block(int32_t max_env, int64_t n_drones, int n_sm);

cudaError_t launch_step(const StepArgs& a, int n_tiles, int block, bool with_obs, int uniform_flags, cudaStream_t s);
// grid: persistent CTAs (0: one per work item)
cudaError_t launch_rollout(const RolloutArgs& a, int block, int uniform_flags, int grid, cudaStream_t s);
int rollout_blocks_per_sm(int block, int uniform_flags, int uniform_N);
cudaError_t launch_obs(const StepArgs& a, int n_tiles, int block, cudaStream_t s);
cudaError_t launch_pid(const PidArgs& a, cudaStream_t s);

}  // namespace mdg
