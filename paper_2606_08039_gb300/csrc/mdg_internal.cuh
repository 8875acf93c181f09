// Internal declarations shared by the host API (mdg_api.cu) and the kernels (mdg_step.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mdg.h"

namespace mdg {

// Index checks of the debug build (compiled with -DMDG_DEBUG): a false condition records
// MDG_STATUS_BOUNDS in the status word and lets the caller skip the access. Release builds
// compile every check to `true`.
#ifdef MDG_DEBUG
#define MDG_CHECK(cond, status) ((cond) ? true : (atomicOr((status), MDG_STATUS_BOUNDS), false))
#else
#define MDG_CHECK(cond, status) true
#endif

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
    float hover_rpm;                  // normalized actions: 0 -> HOVER_RPM
    float alloc_xy, alloc_z;          // inverse mixing: sqrt(2)/L (X) or 2/L (+), and k_f/k_m
    float mix_x[4], mix_y[4];         // inverse mixing signs of tau_x, tau_y per rotor
    int frame_p;                      // 1: + rotor layout (l_sqrt2 then holds L)
    int rk4;                          // 1: fourth-order Runge-Kutta substeps
    int gnd_rotor;                    // 1: Eq. ground at each rotor's height (runtime-flag kernels)
    int dsl;                          // 1: DSL controller (rate-limited setpoints; runtime-flag kernels)
    float sp_step_pos, sp_step_yaw;   // DSL setpoint limits per control period (rate x dt_ctrl)
    float rotor_x[4], rotor_y[4];     // rotor body positions (z = 0)
};

// A launch tile: whole environments packed into one thread block.
// x = first drone, y = drones, z = first environment,
// w = environments (low 16 bits) | kTileAnyDW | kTileWarpLocal.
typedef int4 Tile;
constexpr int kTileEnvMask = 0xffff;
constexpr int kTileAnyDW = 1 << 30;      // some environment of the tile has downwash on
constexpr int kTileWarpLocal = 1 << 29;  // every environment lies inside one warp

// The buffers of mdg_set_randomization, kept in a small device allocation of the handle.
struct RandArgs {
    const float* dr;          // [n_envs][MDG_DR_PARAMS] domain randomization and wind
    float4* motor;            // [n] rotor speeds (the motor lag's state)
    float4* hist;             // [depth][n] actions received (the latency's shift register)
    float4* wind;             // [n_envs][2] wind state
    unsigned long long seed;  // of the wind draws
    int depth;
    const float4* obs_bias;   // [n][3] sticky per-episode observation bias (12 floats per drone), or null
};

// Episode reset (mdg_reset): the init row of the randomization table and the observation bias.
struct ResetArgs {
    float4* state;            // [6][n]
    const float4* nominal;    // [n] x, y, z, yaw
    float4* obs_bias;         // [n][3] or null
    long long n;
    float range_pos, range_att, range_vel;
    float sigma[4];           // bias sigmas: position, roll/pitch/yaw, velocity, body rate
    unsigned long long seed, episode;
};

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
    int obs_host;             // 1: observations go to host memory, written through per-warp staging
    DevConsts c;
    // after the constants, so that their offsets (and the hot kernels' code) stay put; the
    // randomization buffers sit behind one device pointer to keep the argument block small
    float4* setpoints;        // [n] DSL setpoints (x, y, z, yaw) or null
    const RandArgs* rand;     // device copy of the randomization buffers, or null
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
    const int* sched_off;       // static schedule: block b runs sched_items[sched_off[b] .. sched_off[b + 1]),
    const int* sched_items;     // in that order (null: items from the work counter)
};

// The surrogate's parameters as the kernels see them.
struct MlpView {
    float* master;   // FP32 flat parameters
    void* w16;       // bf16 copies (same offsets; bias slots unused)
    int w_off[4], b_off[4];
};

// Per-control-step surrogate kernels (uniform batches).
struct SurrogateArgs {
    StepArgs s;                  // state, action, tables, constants
    void* x;                     // [n_pad][64] bf16 standardised inputs
    const float* y;              // [n_pad][32] standardised outputs of the network
    const float* in_mean;        // [41]
    const float* in_inv_std;     // [41]
    const float* in_lo;          // [41]
    const float* in_hi;          // [41]
    const float* out_mean;       // [13]
    const float* out_std;        // [13]
    float ood_z;
    unsigned* env_flag;          // [n_envs], zeroed before prepare
    int* fallback_list;          // [n_envs]
    int* fallback_count;         // [1], zeroed before prepare
    float* raw;                  // features only: [n][41]
    const float4* rpm;           // features only: [n]
};

struct PidArgs {
    float4* state;
    const float4* waypoints;
    const float4* target_acc;  // [n] feed-forward (x, y, z, -) or null
    float4* setpoints;         // [n] DSL setpoints or null
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

// Camera frames (mdg_render).
struct CamArgs {
    const float4* state;     // [6][n] planes (positions and attitudes read)
    long long n;
    int n_envs;
    const int32_t* env_off;  // [n_envs + 1]
    int uniform_N;           // > 0: every environment has this many drones
    uchar4* rgba;            // [n][48 * 64] or null
    float* depth;            // [n][48 * 64] or null
    int* seg;                // [n][48 * 64] or null
    float semi_a, semi_c;    // the drones' ellipsoid semi-axes (a, a, c)
    int max_env;             // drones of the largest environment (shared-memory size)
    uint32_t* status;        // debug builds: MDG_STATUS_BOUNDS
};
cudaError_t launch_render(const CamArgs& a, cudaStream_t s);

// The step-kernel variant that runs under domain randomization (mdg_set_randomization).
constexpr int kVariantRandomized = 11;

// Action types the kernels accept, and those only the runtime-flag kernels convert.
inline bool valid_env_action(int t) { return t == MDG_ACT_RPM || t == MDG_ACT_PID || (t >= MDG_ACT_RPM_NORM && t <= MDG_ACT_ATTITUDE); }
inline bool valid_action(int t) { return valid_env_action(t) || t == MDG_ACT_MIXED; }
inline bool extended_action(int t) { return t >= MDG_ACT_RPM_NORM && t <= MDG_ACT_ATTITUDE; }
// grid: persistent CTAs (0: one per work item)
cudaError_t launch_rollout(const RolloutArgs& a, int block, int uniform_flags, int grid, cudaStream_t s);
int rollout_blocks_per_sm(const StepArgs& a, int block, int uniform_flags);
cudaError_t launch_features(const SurrogateArgs& a, int n_tiles, int block, cudaStream_t s);
cudaError_t launch_surrogate_prepare(const SurrogateArgs& a, int n_tiles, int block, cudaStream_t s);
cudaError_t launch_surrogate_apply(const SurrogateArgs& a, cudaStream_t s);
cudaError_t launch_surrogate_fallback(const SurrogateArgs& a, cudaStream_t s);

// mdg_mlp.cu
cudaError_t mlp_forward(const MlpView& w, const void* x, int B, float* z_hidden[3], void* h_hidden[3], float* y,
                        const float* target, void* dy, float* loss_acc, cudaStream_t s);
cudaError_t mlp_backward(const MlpView& w, const void* x, int B, float* const z_hidden[3], void* const h_hidden[3],
                         void* dy, void* dz_hidden[3], float* grad, cudaStream_t s);
cudaError_t mlp_adam(const MlpView& w, const float* grad, float* m, float* v, float lr, int step, cudaStream_t s);
cudaError_t mlp_refresh_bf16(const MlpView& w, cudaStream_t s);
cudaError_t mlp_standardize(const float* raw, void* x, long long rows, const float* mean, const float* inv_std,
                            cudaStream_t s);
// db[n] = sum over the M rows of dz[m][n] (bf16 [M][N])
cudaError_t mlp_bias_grad(const void* dz, int M, int N, float* db, cudaStream_t s);

// Scratch of the tcgen05 training pass (batch B <= max_batch rows): the forward pass's
// pre-activations z (FP32 [B][256]) and activations h (bf16 [B][256]) with their transposes hT
// ([256][B]), the output y (FP32 [B][32]) and its gradient dy (bf16 [B][32], transposed dyT
// [32][B]), the hidden gradients dz ([B][256], transposed dzT), the transposed input xT
// ([64][B]) and the transposed weights wT (W2^T, W3^T [256][256], W4^T [256][32], bf16).
struct TrainBuffers {
    float* z[3];
    void* h[3];
    void* hT[3];
    void* dz[3];
    void* dzT[3];
    float* y;
    void* dy;
    void* dyT;
    void* xT;
    const void* wT;
};
// mdg_umma.cu: fused tcgen05 forward, B a multiple of 128, y [B][32]. `img` is the weight
// image of mlp_build_image (mlp_image_bytes() bytes, 16-byte aligned), rebuilt whenever the
// bf16 weights change.
size_t mlp_image_bytes();
cudaError_t mlp_build_image(const MlpView& w, void* img, cudaStream_t s);
cudaError_t mlp_forward_umma(const MlpView& w, const void* img, const void* x, int B, float* y, uint32_t* status,
                             int wait_limit, int spin_limit, cudaStream_t s);
// The surrogate's update of the state by the network's prediction, done in the output stage
// of the paired kernel instead of writing y: for every row g < n whose environment
// (g / uniform_N) is not flagged, p, v, omega += out_mean + out_std * y and the quaternion the
// same, renormalised (the arithmetic of surrogate_apply_kernel). state: the [6][n] planes.
struct MlpApply {
    float4* state;
    long long n;
    int uniform_N;
    const unsigned* env_flag;  // [n_envs]
    const float* out_mean;     // [13]
    const float* out_std;      // [13]
};
// The same with two 128-row tiles in flight per block (one 256-column accumulator each); with
// apply, the state is updated and y is not written.
cudaError_t mlp_forward_umma_pairs(const MlpView& w, const void* img, const void* x, int B, float* y,
                                   uint32_t* status, int wait_limit, int spin_limit, cudaStream_t s,
                                   const MlpApply* apply = nullptr);
// Training on tcgen05: the loss of the standardised targets t ([B][32], columns 13..31
// ignored) added to *loss_acc and every parameter's gradient written to grad (flat FP32
// layout); B a multiple of 128. wT must hold the current weights' transposes.
cudaError_t mlp_grad_umma(const MlpView& w, const TrainBuffers& t, const void* x, int B, const float* target,
                          float* loss_acc, float* grad, uint32_t* status, cudaStream_t s);
cudaError_t mlp_weights_transposed(const MlpView& w, void* wT, cudaStream_t s);
size_t mlp_weights_transposed_elems();

cudaError_t launch_obs(const StepArgs& a, int n_tiles, int block, cudaStream_t s);
cudaError_t launch_reset(const ResetArgs& r, cudaStream_t s);
cudaError_t launch_pid(const PidArgs& a, cudaStream_t s);

}  // namespace mdg

// The handle behind mdg_handle (host side).
struct mdg_ctx {
    int device = 0;
    int32_t n_envs = 0;
    int64_t n_drones = 0;
    int32_t max_env = 0;
    mdg_constants c{};
    mdg::DevConsts dc{};
    mdg_constants cc{};  // the constants as given (host)
    std::vector<int32_t> h_off;
    std::vector<uint8_t> h_flags;
    int32_t* d_off = nullptr;
    uint8_t* d_flags = nullptr;
    uint8_t* d_act = nullptr;
    bool act_set = false;
    bool act_ext = false;  // some environment's type is beyond RPM/PID (runtime-flag kernels)
    float4* d_sp = nullptr;  // caller-owned DSL setpoints (mdg_set_setpoints)
    // caller-owned domain randomization (mdg_set_randomization); dr == nullptr: none
    const float* dr = nullptr;
    mdg::RandArgs* d_rand = nullptr;  // device copy of the buffers (allocated on first attach)
    mdg::RandArgs rand_host = {};     // what d_rand holds (valid while dr != nullptr)
    mdg::Tile* d_tiles = nullptr;
    int n_tiles = 0;
    int block = 0;
    int uniform_N = 0;      // every environment has this many drones (0: mixed sizes)
    int envs_per_tile = 0;
    int uniform_bits = 0;
    int uniform_flags = -1;  // physics subset shared by every environment, -1 if they differ
    uint32_t* d_status = nullptr;
    // rollout work items, built on first use for the current block size, item cap and grid
    int rollout_block = 0;
    int rollout_cap = -1;   // the item cap the items were built for
    int item_cap = 0;       // at most this many drones per work item of an uneven batch (0: the block size)
    int sched = 0;          // MDG_SCHED_DYNAMIC or MDG_SCHED_STATIC
    int sched_grid = 0;     // the grid the static schedule was built for (0: none)
    int* d_sched_off = nullptr;
    int* d_sched_items = nullptr;
    std::vector<double> item_cost;  // host: the chain estimate of every item
    int n_items = 0;
    int4* d_items = nullptr;
    int* d_item_order = nullptr;
    int* d_slot_env = nullptr;
    int* d_slot_goff = nullptr;
    int* d_slot_loff = nullptr;
    int* d_counter = nullptr;
};
