// mdg_step_obs_noalloc: one control step without any device allocation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is owned by
// another allocator (a training framework's caching allocator that has reserved the free
// memory), or a control loop that must not allocate once it runs. They cannot create a
// handle, because mdg_create allocates the batch tables and the status word. This entry
// point keeps those tables in a file-scope static device array instead, so the only
// device memory it touches is that array and the caller's own buffers.
//
// The array g_scratch is reserved in every GPU that loads the library's device code, for
// the life of the process; with lazy module loading (the CUDA default) that happens at the
// first call on a device, which therefore needs about 353 KiB of free device memory plus the
// library's code. Every call shares the array and it keeps the last call's contents, so
// calls that overlap on the GPU (on different streams, or from different host threads) race.
// A call made while its stream is being captured into a CUDA graph is refused: the tables
// are uploaded from a host staging buffer that the next call overwrites, so a replayed
// graph would pair one batch's sizes with another batch's tables.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "mdg.h"
#include "mdg_internal.cuh"

namespace {

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t kOffStatus = 0;                                              // uint32 [2]
constexpr size_t kOffEnvOff = 256;                                            // int32 [max_envs + 1]
constexpr size_t kEnvOffBytes = ((4 * (MDG_NOALLOC_MAX_ENVS + 1) + 255) / 256) * 256;
constexpr size_t kOffFlags = kOffEnvOff + kEnvOffBytes;                       // uint8 [max_envs]
constexpr size_t kOffAct = kOffFlags + MDG_NOALLOC_MAX_ENVS;                  // uint8 [max_envs]
constexpr size_t kOffTiles = kOffAct + MDG_NOALLOC_MAX_ENVS;                  // int4 [max_envs]
constexpr size_t kScratchBytes = kOffTiles + 16 * (size_t)MDG_NOALLOC_MAX_ENVS;
static_assert(kScratchBytes == MDG_NOALLOC_SCRATCH_BYTES, "scratch layout does not match mdg.h");
static_assert(kOffTiles % 256 == 0 && kOffFlags % 256 == 0, "scratch offsets must stay aligned");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host staging copy of the tables (static storage, reused by every call under g_lock).
unsigned char g_stage[kScratchBytes];
std::mutex g_lock;
bool g_loaded[64] = {};  // the device has given g_scratch's address once (its module is loaded)

// Records the message for mdg_last_error() and returns the code.
int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    mdg::set_last_error(buf);
    return code;
}

// The device address of g_scratch on the current device, looked up on every call with the
// device current (in host code g_scratch names a host-side stand-in, not device memory). A
// cached address would outlive the context it belongs to: after cudaDeviceReset the next
// call runs in a new context, where the array has been reserved again, maybe elsewhere. The
// first lookup on a device loads the library's device code and reserves the array there.
int scratch_address(int dev, void** out)
{
    if (dev < 0 || dev >= 64) return fail(MDG_ERR_UNSUPPORTED, "mdg_step_obs_noalloc: device %d out of range", dev);
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        if (!g_loaded[dev])
            return fail(MDG_ERR_CUDA,
                        "mdg_step_obs_noalloc: first call on device %d: loading the library's device code and its "
                        "%d-byte static array failed (%s); make the first call before another allocator reserves "
                        "the device's free memory",
                        dev, (int)kScratchBytes, cudaGetErrorString(e));
        return fail(MDG_ERR_CUDA, "mdg_step_obs_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    }
    g_loaded[dev] = true;
    *out = p;
    return MDG_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int mdg_step_obs_noalloc(const mdg_constants* c, int32_t n_envs, const int32_t* drones_per_env,
                                    const uint32_t* model_flags, const uint8_t* action_types, float* state,
                                    const float* action, int32_t action_type, int32_t n_substeps, float* kin,
                                    int32_t* nbr_idx, float* nbr_rel, uint32_t* status_out, void* stream)
{
    // ---- arguments (host only, nothing launched yet)
    if (n_envs < 0) return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: n_envs < 0");
    if (n_envs > MDG_NOALLOC_MAX_ENVS)
        return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: n_envs = %d exceeds the static maximum of %d environments",
                    n_envs, MDG_NOALLOC_MAX_ENVS);
    if (n_envs > 0 && (!drones_per_env || !model_flags))
        return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: drones_per_env and model_flags are required");
    if (!mdg::valid_action(action_type))
        return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: unknown action_type %d", action_type);
    if (action_type == MDG_ACT_MIXED && n_envs > 0 && !action_types)
        return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: MDG_ACT_MIXED needs action_types");
    if (n_substeps < 1) return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: n_substeps = %d < 1", n_substeps);
    mdg_constants cc;
    if (c) cc = *c;
    else mdg_constants_cf2x(&cc);
    std::string why;
    if (!mdg::constants_valid(cc, why)) return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: %s", why.c_str());
    if (cc.controller == MDG_CTRL_DSL)
        return fail(MDG_ERR_UNSUPPORTED, "mdg_step_obs_noalloc: the DSL controller needs a handle's setpoints");
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    const cudaError_t cap = cudaStreamIsCapturing((cudaStream_t)stream, &capturing);
    if (cap != cudaSuccess)
        return fail(MDG_ERR_CUDA, "mdg_step_obs_noalloc: cudaStreamIsCapturing: %s", cudaGetErrorString(cap));
    if (capturing != cudaStreamCaptureStatusNone)
        return fail(MDG_ERR_UNSUPPORTED,
                    "mdg_step_obs_noalloc: the stream is being captured; the call uploads its tables from a host "
                    "buffer that the next call overwrites, so it cannot be replayed from a graph");

    std::lock_guard<std::mutex> lock(g_lock);
    int32_t* off = reinterpret_cast<int32_t*>(g_stage + kOffEnvOff);
    uint8_t* flg = g_stage + kOffFlags;
    uint8_t* act = g_stage + kOffAct;
    off[0] = 0;
    int64_t total = 0;
    int32_t max_env = 0;
    bool ext = mdg::extended_action(action_type);
    for (int32_t e = 0; e < n_envs; ++e) {
        const int32_t N = drones_per_env[e];
        if (N < 0 || N > MDG_MAX_ENV_DRONES)
            return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: drones_per_env[%d] = %d outside [0, %d]", e, N,
                        MDG_MAX_ENV_DRONES);
        if (model_flags[e] & ~(MDG_GND | MDG_DRAG | MDG_DW))
            return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: model_flags[%d] has unknown bits", e);
        if (action_type == MDG_ACT_MIXED) {
            if (!mdg::valid_env_action(action_types[e]))
                return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: action_types[%d] is not an action type", e);
            ext = ext || mdg::extended_action(action_types[e]);
        }
        total += N;
        if (total > 0x7fffffffLL) return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: more than 2^31 - 1 drones");
        off[e + 1] = (int32_t)total;
        flg[e] = (uint8_t)model_flags[e];
        act[e] = action_type == MDG_ACT_MIXED ? action_types[e] : (uint8_t)action_type;
        if (N > max_env) max_env = N;
    }
    if (total == 0) return MDG_OK;
    const void* req[] = {state, action, nbr_idx};
    const char* names[] = {"state", "action", "nbr_idx"};
    for (int i = 0; i < 3; ++i) {
        if (i == 2 && !kin) break;
        if (!req[i]) return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: %s is NULL", names[i]);
        if (!aligned16(req[i])) return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: %s is not 16-byte aligned", names[i]);
    }
    if (kin && !aligned16(kin)) return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: kin is not 16-byte aligned");
    if (nbr_rel && !aligned16(nbr_rel)) return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: nbr_rel is not 16-byte aligned");
    if (status_out && (reinterpret_cast<uintptr_t>(status_out) & 3u))
        return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: status_out is not 4-byte aligned");

    // ---- tiles and the per-batch facts the kernels branch on (host, static staging)
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return fail(MDG_ERR_CUDA, "mdg_step_obs_noalloc: cudaGetDevice: %s", cudaGetErrorString(ce));
    void* scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc != MDG_OK) return rc;
    int n_sm = 152;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int block = mdg::default_block(max_env, total, n_sm > 0 ? n_sm : 152);
    // greedy packing of whole environments into tiles (the handle API's rule), written
    // straight into the staging area: at most one tile per environment
    mdg::Tile* tiles = reinterpret_cast<mdg::Tile*>(g_stage + kOffTiles);
    int n_tiles = 0;
    int uniform_bits = mdg::kTileWarpLocal, any_dw = 0;
    for (int e = 0; e < n_envs;) {
        const int e0 = e;
        while (e < n_envs && (off[e + 1] - off[e0]) <= block && (e + 1 - e0) <= block) ++e;
        if (e == e0) return fail(MDG_ERR_ARG, "mdg_step_obs_noalloc: environment %d does not fit a block", e0);
        mdg::Tile t;
        t.x = off[e0];
        t.y = off[e] - off[e0];
        t.z = e0;
        t.w = e - e0;
        bool dw = false, local = true;
        for (int k = e0; k < e; ++k) {
            const int ls = off[k] - off[e0], N = off[k + 1] - off[k];
            if (N > 0 && (flg[k] & MDG_DW)) dw = true;
            if (N > 0 && (ls >> 5) != ((ls + N - 1) >> 5)) local = false;
        }
        if (dw) {
            t.w |= mdg::kTileAnyDW;
            any_dw = mdg::kTileAnyDW;
        }
        if (local) t.w |= mdg::kTileWarpLocal;
        else uniform_bits = 0;
        if (t.y > 0) tiles[n_tiles++] = t;
    }
    bool uniform = n_envs > 0;
    int uniform_flags = n_envs > 0 ? flg[0] : -1;
    for (int e = 0; e < n_envs; ++e) {
        if (off[e + 1] - off[e] != max_env) uniform = false;
        if (flg[e] != flg[0]) uniform_flags = -1;
    }
    if (ext) uniform_flags = 8;  // action types beyond RPM/PID: the runtime-flag kernels
    uint32_t* st = reinterpret_cast<uint32_t*>(g_stage + kOffStatus);
    st[0] = 0u;            // status bits start clear
    st[1] = 0xffffffffu;   // no offending drone yet

    // ---- upload the tables and the cleared status word into the static array
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* d = static_cast<unsigned char*>(scratch);
    const size_t env_bytes = 4 * (size_t)(n_envs + 1);
    if ((ce = cudaMemcpyAsync(d + kOffStatus, g_stage + kOffStatus, 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (ce = cudaMemcpyAsync(d + kOffEnvOff, g_stage + kOffEnvOff, env_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (ce = cudaMemcpyAsync(d + kOffFlags, g_stage + kOffFlags, (size_t)n_envs, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (ce = cudaMemcpyAsync(d + kOffAct, g_stage + kOffAct, (size_t)n_envs, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (ce = cudaMemcpyAsync(d + kOffTiles, g_stage + kOffTiles, 16 * (size_t)n_tiles, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
        return fail(MDG_ERR_CUDA, "mdg_step_obs_noalloc: upload: %s", cudaGetErrorString(ce));

    // ---- the step kernel on the static tables
    mdg::StepArgs a{};
    a.state = reinterpret_cast<float4*>(state);
    a.action = reinterpret_cast<const float4*>(action);
    a.kin = kin;
    a.nbr_idx = reinterpret_cast<int4*>(nbr_idx);
    a.nbr_rel = kin ? nbr_rel : nullptr;
    a.tiles = reinterpret_cast<const mdg::Tile*>(d + kOffTiles);
    a.env_off = reinterpret_cast<const int32_t*>(d + kOffEnvOff);
    a.env_flags = d + kOffFlags;
    a.env_act = d + kOffAct;
    a.status = reinterpret_cast<uint32_t*>(d + kOffStatus);
    a.n = total;
    a.n_sub = n_substeps;
    a.act_type = action_type;
    a.n_envs = n_envs;
    a.uniform_N = uniform ? max_env : 0;
    a.envs_per_tile = uniform ? block / max_env : 0;
    a.uniform_bits = any_dw | uniform_bits;
    a.c = mdg::make_dev_consts(cc);
    ce = mdg::launch_step(a, n_tiles, block, kin != nullptr, uniform_flags, s);
    if (ce != cudaSuccess) return fail(MDG_ERR_CUDA, "mdg_step_obs_noalloc: launch: %s", cudaGetErrorString(ce));
    if (status_out) {
        ce = cudaMemcpyAsync(status_out, d + kOffStatus, 8, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess)
            return fail(MDG_ERR_CUDA, "mdg_step_obs_noalloc: status copy: %s", cudaGetErrorString(ce));
    }
    return MDG_OK;
}
